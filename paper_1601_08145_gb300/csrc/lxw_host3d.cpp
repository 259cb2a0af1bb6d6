// lxw_host3d.cpp -- C ABI of the 3D Cartesian FP64 form (lxw3_*): tables,
// solver object, step / run / profile.  The kernels are in lxw_kernels3d.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lxw.h"
#include "lxw_internal3d.h"

using namespace lxw;

struct lxw_solver3 {
  int nx = 0, ny = 0, nz = 0, N = 0, deg = 0, ML = 0, NF = 0, NPJ = 0;
  double box[6] = {0, 0, 0, 0, 0, 0};
  int bc[6] = {0, 0, 0, 0, 0, 0};
  lxw_options opt{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;   // graphs are captured here (the caller's stream may be the legacy one)
  Mesh3 dm{};
  Work3 dw{};
  double* jw = nullptr;          // [NPJ] projection weights (device)
  double* jphi = nullptr;        // [NPJ][ML] projection basis (device)
  std::vector<double> pj;        // projection points on the reference cube [NPJ][3]
  std::vector<void*> allocs;
  cudaGraphExec_t graph = nullptr;   // one step without diagnostics
  double graph_cfl = -1.0;           // ... captured for this CFL number
  double* graph_q = nullptr;         // ... and this state
  cudaEvent_t ev[8] = {};
  ~lxw_solver3() {
    if (graph) cudaGraphExecDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
    for (void* p : allocs) cudaFree(p);
  }
};

namespace {

lxw_status fail3(lxw_status st, const std::string& msg) {
  set_last_error(msg.c_str());
  return st;
}

#define LXW3_CUDA(call)                                                                                    \
  do {                                                                                                     \
    cudaError_t e_ = (call);                                                                               \
    if (e_ != cudaSuccess) return fail3(LXW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int modes3(int deg) { return (deg + 1) * (deg + 2) * (deg + 3) / 6; }

// exponents (a, b, c) of each mode: total degree ascending, then a, then b descending
void exponents3(int deg, std::vector<int>& abc) {
  abc.clear();
  for (int t = 0; t <= deg; ++t)
    for (int a = t; a >= 0; --a)
      for (int b = t - a; b >= 0; --b) { abc.push_back(a); abc.push_back(b); abc.push_back(t - a - b); }
}

// basis and reference gradient at one point of the reference cube
void basis3(int deg, const std::vector<int>& abc, const double r[3], double* phi, double* grad /* [3][ML] or null */) {
  const int ML = modes3(deg);
  double v[3][4], d[3][4];
  for (int ax = 0; ax < 3; ++ax)
    for (int n = 0; n <= deg; ++n) host_legendre_norm(n, r[ax], v[ax][n], d[ax][n]);
  for (int l = 0; l < ML; ++l) {
    const int a = abc[3 * l], b = abc[3 * l + 1], c = abc[3 * l + 2];
    phi[l] = v[0][a] * v[1][b] * v[2][c];
    if (grad) {
      grad[0 * ML + l] = d[0][a] * v[1][b] * v[2][c];
      grad[1 * ML + l] = v[0][a] * d[1][b] * v[2][c];
      grad[2 * ML + l] = v[0][a] * v[1][b] * d[2][c];
    }
  }
}

void make_tables3(int deg, Tables3& t, std::vector<double>& pj, std::vector<double>& jw, std::vector<double>& jphi) {
  std::memset(&t, 0, sizeof(t));
  const int ML = modes3(deg), n = deg + 1, NQ = n * n * n, NF = n * n;
  std::vector<int> abc;
  exponents3(deg, abc);
  double g[8], gw[8];
  host_gauss_legendre(n, g, gw);
  // interior points and weights (sum 1)
  std::vector<double> pts;
  for (int c = 0; c < n; ++c)
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        const int k = (c * n + b) * n + a;
        t.qw[k] = gw[a] * gw[b] * gw[c] / 8.0;
        pts.insert(pts.end(), {g[a], g[b], g[c]});
      }
  for (int tt = 0; tt < n; ++tt)
    for (int u = 0; u < n; ++u) t.fw[tt * n + u] = gw[u] * gw[tt] / 4.0;
  // face points: face k on axis d = k / 2 at xi_d = -1 (k even) or +1 (k odd)
  for (int k = 0; k < 6; ++k) {
    const int d = k / 2, d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
    for (int tt = 0; tt < n; ++tt)
      for (int u = 0; u < n; ++u) {
        double r[3];
        r[d] = (k & 1) ? 1.0 : -1.0; r[d1] = g[u]; r[d2] = g[tt];
        pts.insert(pts.end(), {r[0], r[1], r[2]});
      }
  }
  const int NPT = NQ + 6 * NF;
  std::vector<double> grad(3 * ML);
  for (int p = 0; p < NPT; ++p) {
    basis3(deg, abc, &pts[3 * p], t.phi[p], p < NQ ? grad.data() : nullptr);
    if (p < NQ)
      for (int ax = 0; ax < 3; ++ax)
        for (int l = 0; l < ML; ++l) t.dref[ax][p][l] = grad[ax * ML + l];
  }
  // D_d[m][l] = (1/8) Int d_d phi_m phi_l (exact with n points per direction),
  // W_d[k][l] = qw_k sum_m phi_m(x_k) D_d[m][l]
  for (int ax = 0; ax < 3; ++ax) {
    std::vector<double> D(ML * ML, 0.0);
    for (int m = 0; m < ML; ++m)
      for (int l = 0; l < ML; ++l) {
        double s = 0.0;
        for (int k = 0; k < NQ; ++k) s += t.qw[k] * t.dref[ax][k][m] * t.phi[k][l];
        D[m * ML + l] = s;
      }
    for (int k = 0; k < NQ; ++k)
      for (int l = 0; l < ML; ++l) {
        double s = 0.0;
        for (int m = 0; m < ML; ++m) s += t.phi[k][m] * D[m * ML + l];
        t.W[ax][k][l] = t.qw[k] * s;
      }
  }
  // projection rule: deg + 3 points per direction
  const int nj = deg + 3;
  double gj[8], gjw[8];
  host_gauss_legendre(nj, gj, gjw);
  pj.clear(); jw.clear(); jphi.clear();
  std::vector<double> ph(ML);
  for (int c = 0; c < nj; ++c)
    for (int b = 0; b < nj; ++b)
      for (int a = 0; a < nj; ++a) {
        const double r[3] = {gj[a], gj[b], gj[c]};
        pj.insert(pj.end(), {r[0], r[1], r[2]});
        jw.push_back(gjw[a] * gjw[b] * gjw[c] / 8.0);
        basis3(deg, abc, r, ph.data(), nullptr);
        jphi.insert(jphi.end(), ph.begin(), ph.end());
      }
}

}  // namespace

extern "C" {

lxw_status lxw3_solver_create(int nx, int ny, int nz, const double box[6], const int bc[6], int degree,
                              const lxw_options* optp, void* stream, lxw_solver3** out) {
  if (!out || !box || !bc) return fail3(LXW_ERR_ARG, "lxw3_solver_create: null argument");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return fail3(LXW_ERR_ARG, "lxw3_solver_create: nx, ny, nz must be >= 1");
  if ((long long)nx * ny * nz > (1ll << 30)) return fail3(LXW_ERR_ARG, "lxw3_solver_create: more than 2^30 cells");
  if (degree < 1 || degree > 2) return fail3(LXW_ERR_ARG, "lxw3_solver_create: degree must be 1 or 2");
  for (int d = 0; d < 3; ++d)
    if (!(box[2 * d + 1] > box[2 * d])) return fail3(LXW_ERR_ARG, "lxw3_solver_create: empty box");
  for (int k = 0; k < 6; ++k)
    if (bc[k] != LXW_BC_PERIODIC && bc[k] != LXW_BC_REFLECT && bc[k] != LXW_BC_TRANSPARENT)
      return fail3(LXW_ERR_ARG, "lxw3_solver_create: boundary codes are periodic, reflective or transparent");
  for (int d = 0; d < 3; ++d)
    if ((bc[2 * d] == LXW_BC_PERIODIC) != (bc[2 * d + 1] == LXW_BC_PERIODIC))
      return fail3(LXW_ERR_ARG, "lxw3_solver_create: periodic sides must be paired");
  lxw_options opt;
  if (optp) opt = *optp; else lxw_options_default(&opt);
  if (!(opt.gamma > 1.0)) return fail3(LXW_ERR_ARG, "lxw3_solver_create: gamma must exceed 1");
  if (opt.precision != LXW_PREC_FP64) return fail3(LXW_ERR_ARG, "lxw3_solver_create: the 3D form is FP64 only");
  if (opt.moment_exact || (opt.ck_order != 0 && opt.ck_order != 3))
    return fail3(LXW_ERR_ARG, "lxw3_solver_create: moment_exact and ck_order 4 are 2D options");
  if (opt.block_threads <= 0) opt.block_threads = 128;
  if (opt.block_threads % 32 || opt.block_threads > 128)
    return fail3(LXW_ERR_ARG, "lxw3_solver_create: block_threads must be a multiple of 32, at most 128");
  lxw_solver3* s = new (std::nothrow) lxw_solver3;
  if (!s) return fail3(LXW_ERR_NOMEM, "lxw3_solver_create: host allocation failed");
  s->nx = nx; s->ny = ny; s->nz = nz; s->N = nx * ny * nz; s->deg = degree;
  s->ML = modes3(degree); s->NF = (degree + 1) * (degree + 1);
  std::memcpy(s->box, box, sizeof(s->box));
  std::memcpy(s->bc, bc, sizeof(s->bc));
  s->opt = opt;
  s->stream = (cudaStream_t)stream;
  Tables3 t;
  std::vector<double> jw, jphi;
  make_tables3(degree, t, s->pj, jw, jphi);
  s->NPJ = (int)jw.size();
  if (upload_tables3(degree, t)) { delete s; return fail3(LXW_ERR_CUDA, "lxw3_solver_create: table upload failed"); }
  const size_t N = s->N;
  auto dalloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    s->allocs.push_back(p);
    return p;
  };
  int* nbr = (int*)dalloc(sizeof(int) * 6 * N);
  s->dw.trace = (double*)dalloc(sizeof(double) * 6 * s->NF * 10 * N);
  s->dw.flux = (double*)dalloc(sizeof(double) * 60 * N);
  s->dw.prop = (double*)dalloc(sizeof(double) * 6 * N);
  s->dw.smax = (unsigned long long*)dalloc(sizeof(unsigned long long));
  s->dw.status = (unsigned int*)dalloc(sizeof(unsigned int));
  s->dw.diag = (Diag3Block*)dalloc(sizeof(Diag3Block));
  s->jw = (double*)dalloc(sizeof(double) * jw.size());
  s->jphi = (double*)dalloc(sizeof(double) * jphi.size());
  if (!nbr || !s->dw.trace || !s->dw.flux || !s->dw.prop || !s->dw.smax || !s->dw.status || !s->dw.diag || !s->jw ||
      !s->jphi) {
    delete s;
    return fail3(LXW_ERR_NOMEM, "lxw3_solver_create: device allocation failed");
  }
  // neighbours [6][N]: faces x-, x+, y-, y+, z-, z+
  std::vector<int> hn(6 * N);
  const int n3[3] = {nx, ny, nz};
  for (int iz = 0; iz < nz; ++iz)
    for (int iy = 0; iy < ny; ++iy)
      for (int ix = 0; ix < nx; ++ix) {
        const size_t i = ((size_t)iz * ny + iy) * nx + ix;
        for (int k = 0; k < 6; ++k) {
          int cc[3] = {ix, iy, iz};
          const int d = k / 2;
          cc[d] += (k & 1) ? 1 : -1;
          int v;
          if (cc[d] < 0 || cc[d] >= n3[d]) {
            if (bc[k] == LXW_BC_PERIODIC) {
              cc[d] = (cc[d] + n3[d]) % n3[d];
              v = (cc[2] * ny + cc[1]) * nx + cc[0];
            } else {
              v = -1 - bc[k];
            }
          } else {
            v = (cc[2] * ny + cc[1]) * nx + cc[0];
          }
          hn[(size_t)k * N + i] = v;
        }
      }
  cudaError_t e = cudaMemcpy(nbr, hn.data(), sizeof(int) * hn.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->jw, jw.data(), sizeof(double) * jw.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->jphi, jphi.data(), sizeof(double) * jphi.size(), cudaMemcpyHostToDevice);
  for (int k = 0; k < 8 && e == cudaSuccess; ++k) e = cudaEventCreate(&s->ev[k]);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete s;
    return fail3(LXW_ERR_CUDA, std::string("lxw3_solver_create: ") + cudaGetErrorString(e));
  }
  s->dm.N = s->N; s->dm.nx = nx; s->dm.ny = ny; s->dm.nz = nz;
  for (int d = 0; d < 3; ++d) s->dm.h[d] = (box[2 * d + 1] - box[2 * d]) / n3[d];
  s->dm.vol = s->dm.h[0] * s->dm.h[1] * s->dm.h[2];
  const double surf = 2.0 * (s->dm.h[0] * s->dm.h[1] + s->dm.h[1] * s->dm.h[2] + s->dm.h[0] * s->dm.h[2]);
  s->dm.hmin = 3.0 * s->dm.vol / surf;
  s->dm.nbr = nbr;
  *out = s;
  return LXW_OK;
}

void lxw3_solver_destroy(lxw_solver3* s) { delete s; }

lxw_status lxw3_solver_info(const lxw_solver3* s, int* n_elements, int* n_modes, int* n_proj_points) {
  if (!s) return fail3(LXW_ERR_ARG, "lxw3_solver_info: null solver");
  if (n_elements) *n_elements = s->N;
  if (n_modes) *n_modes = s->ML;
  if (n_proj_points) *n_proj_points = s->NPJ;
  return LXW_OK;
}

lxw_status lxw3_projection_points(const lxw_solver3* s, double* xyz_host) {
  if (!s || !xyz_host) return fail3(LXW_ERR_ARG, "lxw3_projection_points: null argument");
  for (int iz = 0; iz < s->nz; ++iz)
    for (int iy = 0; iy < s->ny; ++iy)
      for (int ix = 0; ix < s->nx; ++ix) {
        const size_t i = ((size_t)iz * s->ny + iy) * s->nx + ix;
        const double o[3] = {s->box[0] + (ix + 0.5) * s->dm.h[0], s->box[2] + (iy + 0.5) * s->dm.h[1],
                             s->box[4] + (iz + 0.5) * s->dm.h[2]};
        for (int p = 0; p < s->NPJ; ++p)
          for (int d = 0; d < 3; ++d) xyz_host[(i * s->NPJ + p) * 3 + d] = o[d] + 0.5 * s->dm.h[d] * s->pj[3 * p + d];
      }
  return LXW_OK;
}

lxw_status lxw3_project(lxw_solver3* s, const double* prim_dev, double* Q_dev) {
  if (!s || !prim_dev || !Q_dev) return fail3(LXW_ERR_ARG, "lxw3_project: null argument");
  if (launch_project3(s->deg, s->N, s->NPJ, s->opt.gamma, s->jw, s->jphi, prim_dev, Q_dev, s->stream))
    return fail3(LXW_ERR_CUDA, "lxw3_project: launch failed");
  return LXW_OK;
}

int lxw3_step_launches(const lxw_solver3* s) { return s ? step3_launch_count(0, s->opt.shock_limiter) : 0; }

}  // extern "C"

namespace {

Args3 make_args3(const lxw_solver3* s, double dt, double cfl, int want_diag, double* theta_face) {
  Args3 a{};
  a.dt_in = dt; a.cfl = cfl; a.gamma = s->opt.gamma; a.eps0 = s->opt.eps0; a.alpha0 = s->opt.alpha0;
  a.shock_limiter = s->opt.shock_limiter; a.llf_global = s->opt.llf_global; a.want_diag = want_diag;
  a.theta_face = theta_face;
  return a;
}

// status bits of the last step -> return code
lxw_status status3(unsigned st, const char* who) {
  if (st & LXW_ST_NONPOSITIVE) return fail3(LXW_ERR_NONPOSITIVE, std::string(who) + ": non-positive cell average at step start");
  if (st & LXW_ST_CFL) return fail3(LXW_ERR_CFL, std::string(who) + ": Gamma^rho < 0 (dt above the low-order CFL bound)");
  if (st & LXW_ST_NAN) return fail3(LXW_ERR_NAN, std::string(who) + ": non-finite state");
  return LXW_OK;
}

// diagnostics of the step just enqueued (synchronises)
lxw_status read_diag3(lxw_solver3* s, const Args3& a, lxw_diag3* d, const char* who) {
  Diag3Block h{};
  unsigned long long sm = 0;
  unsigned st = 0;
  LXW3_CUDA(cudaMemcpyAsync(&h, s->dw.diag, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
  LXW3_CUDA(cudaMemcpyAsync(&sm, s->dw.smax, sizeof(sm), cudaMemcpyDeviceToHost, s->stream));
  LXW3_CUDA(cudaMemcpyAsync(&st, s->dw.status, sizeof(st), cudaMemcpyDeviceToHost, s->stream));
  LXW3_CUDA(cudaStreamSynchronize(s->stream));
  if (d) {
    auto unob = [](unsigned long long b) {
      b = (b & 0x8000000000000000ull) ? (b & 0x7fffffffffffffffull) : ~b;
      double x;
      std::memcpy(&x, &b, sizeof(x));
      return x;
    };
    std::memset(d, 0, sizeof(*d));
    std::memcpy(&d->s, &sm, sizeof(double));
    d->dt = a.dt_in > 0.0 ? a.dt_in : a.cfl * s->dm.hmin / d->s;
    d->min_rho = unob(h.minr); d->min_p = unob(h.minp);
    d->mass = h.sum[0]; d->momx = h.sum[1]; d->momy = h.sum[2]; d->momz = h.sum[3]; d->energy = h.sum[4];
    d->n_mom = (double)h.nmom; d->n_face = (double)h.nface; d->n_sc = (double)h.nsc;
    d->status = (int)st;
  }
  return status3(st, who);
}

}  // namespace

extern "C" {

lxw_status lxw3_step(lxw_solver3* s, double* Q_dev, double dt, double cfl, lxw_diag3* diag_host,
                     double* theta_face_dev) {
  if (!s || !Q_dev) return fail3(LXW_ERR_ARG, "lxw3_step: null argument");
  if (!(dt > 0.0) && !(cfl > 0.0)) return fail3(LXW_ERR_ARG, "lxw3_step: need dt > 0 or cfl > 0");
  const Args3 a = make_args3(s, dt, cfl, 1, theta_face_dev);
  if (launch_step3(s->deg, s->dm, s->dw, Q_dev, a, s->stream, s->opt.block_threads, nullptr, 99))
    return fail3(LXW_ERR_CUDA, "lxw3_step: launch failed");
  return read_diag3(s, a, diag_host, "lxw3_step");
}

lxw_status lxw3_run(lxw_solver3* s, double* Q_dev, int nsteps, double cfl, lxw_diag3* diag_host) {
  if (!s || !Q_dev || nsteps < 1 || !(cfl > 0.0)) return fail3(LXW_ERR_ARG, "lxw3_run: bad argument");
  // steps without diagnostics replay one captured graph; the last step reports
  const Args3 a = make_args3(s, 0.0, cfl, 0, nullptr);
  if (s->graph && (s->graph_cfl != cfl || s->graph_q != Q_dev)) {
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  if (nsteps > 1 && !s->graph) {
    cudaGraph_t g = nullptr;
    LXW3_CUDA(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = launch_step3(s->deg, s->dm, s->dw, Q_dev, a, s->cap_stream, s->opt.block_threads, nullptr, 99);
    cudaError_t e = cudaStreamEndCapture(s->cap_stream, &g);
    if (rc || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return fail3(LXW_ERR_CUDA, "lxw3_run: graph capture failed");
    }
    e = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail3(LXW_ERR_CUDA, "lxw3_run: graph instantiation failed");
    s->graph_cfl = cfl;
    s->graph_q = Q_dev;
  }
  for (int k = 0; k + 1 < nsteps; ++k) LXW3_CUDA(cudaGraphLaunch(s->graph, s->stream));
  return lxw3_step(s, Q_dev, 0.0, cfl, diag_host, nullptr);
}

lxw_status lxw3_profile_step(lxw_solver3* s, double* Q_dev, double cfl, float* ms) {
  if (!s || !Q_dev || !ms || !(cfl > 0.0)) return fail3(LXW_ERR_ARG, "lxw3_profile_step: bad argument");
  const Args3 a = make_args3(s, 0.0, cfl, 0, nullptr);
  if (launch_step3(s->deg, s->dm, s->dw, Q_dev, a, s->stream, s->opt.block_threads, (void**)s->ev, 99))
    return fail3(LXW_ERR_CUDA, "lxw3_profile_step: launch failed");
  LXW3_CUDA(cudaEventSynchronize(s->ev[5]));
  for (int k = 0; k < 5; ++k) LXW3_CUDA(cudaEventElapsedTime(&ms[k], s->ev[k], s->ev[k + 1]));
  return LXW_OK;
}

}  // extern "C"
