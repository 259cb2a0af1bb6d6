// lxw_host3d.cpp -- C ABI of the 3D FP64 forms (lxw3_*) on Cartesian boxes
// of hexahedra and on tetrahedral meshes: tables, mesh ingestion, solver
// object, step / run / profile.  The kernels are in lxw_kernels3d.cu
// (hexahedra) and lxw_kernels3t.cu (tetrahedra).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lxw.h"
#include "lxw_internal3d.h"

using namespace lxw;

struct lxw_solver3 {
  int kind = 0;                  // 0 hexahedra (Cartesian box), 1 tetrahedra
  int E = 6;                     // faces per element
  int nx = 0, ny = 0, nz = 0, N = 0, deg = 0, ML = 0, NF = 0, NPJ = 0;
  double hmin = 0.0;
  double box[6] = {0, 0, 0, 0, 0, 0};
  int bc[6] = {0, 0, 0, 0, 0, 0};
  lxw_options opt{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;   // graphs are captured here (the caller's stream may be the legacy one)
  Mesh3 dm{};
  Mesh3T tm{};
  std::vector<double> org, jac;  // tetrahedra: vertex 0 [N][3] and d x / d r [N][9] (host)
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
  for (int p = 0; p < NPT; ++p)
    for (int l = 0; l < ML; ++l) t.phimax[l] = std::max(t.phimax[l], std::fabs(t.phi[p][l]));
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

// options of the 3D forms, validated (null: the defaults)
lxw_status options3(const lxw_options* optp, const char* who, lxw_options& opt) {
  if (optp) opt = *optp; else lxw_options_default(&opt);
  const std::string w(who);
  if (!(opt.gamma > 1.0)) return fail3(LXW_ERR_ARG, w + ": gamma must exceed 1");
  if (opt.precision != LXW_PREC_FP64 && opt.precision != LXW_PREC_MIXED)
    return fail3(LXW_ERR_ARG, w + ": the 3D forms are FP64 or mixed (FP32 Cauchy-Kovalevskaya kernel)");
  if (opt.moment_exact || (opt.ck_order != 0 && opt.ck_order != 3))
    return fail3(LXW_ERR_ARG, w + ": moment_exact and ck_order 4 are 2D options");
  if (opt.block_threads <= 0) opt.block_threads = 128;
  if (opt.block_threads % 32 || opt.block_threads > 128)
    return fail3(LXW_ERR_ARG, w + ": block_threads must be a multiple of 32, at most 128");
  return LXW_OK;
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
  if (lxw_status st = options3(optp, "lxw3_solver_create", opt)) return st;
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
  s->dw.fbar = (double*)dalloc(sizeof(double) * 15 * N);
  s->dw.smax = (unsigned long long*)dalloc(sizeof(unsigned long long));
  s->dw.status = (unsigned int*)dalloc(sizeof(unsigned int));
  s->dw.diag = (Diag3Block*)dalloc(sizeof(Diag3Block));
  s->jw = (double*)dalloc(sizeof(double) * jw.size());
  s->jphi = (double*)dalloc(sizeof(double) * jphi.size());
  if (!nbr || !s->dw.trace || !s->dw.flux || !s->dw.prop || !s->dw.fbar || !s->dw.smax || !s->dw.status || !s->dw.diag || !s->jw ||
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
  s->hmin = s->dm.hmin;
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
  if (s->kind == 1) {
    for (size_t i = 0; i < (size_t)s->N; ++i)
      for (int p = 0; p < s->NPJ; ++p) {
        const double* J = &s->jac[9 * i];
        const double* r = &s->pj[3 * p];
        for (int d = 0; d < 3; ++d)
          xyz_host[(i * s->NPJ + p) * 3 + d] = s->org[3 * i + d] + J[3 * d] * r[0] + J[3 * d + 1] * r[1] + J[3 * d + 2] * r[2];
      }
    return LXW_OK;
  }
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

int lxw3_faces_per_element(const lxw_solver3* s) { return s ? s->E : 0; }

}  // extern "C"

namespace {

Args3 make_args3(const lxw_solver3* s, double dt, double cfl, int want_diag, double* theta_face) {
  Args3 a{};
  a.dt_in = dt; a.cfl = cfl; a.gamma = s->opt.gamma; a.eps0 = s->opt.eps0; a.alpha0 = s->opt.alpha0;
  a.shock_limiter = s->opt.shock_limiter; a.llf_global = s->opt.llf_global; a.want_diag = want_diag;
  a.theta_face = theta_face;
  a.ck_fp32 = s->opt.precision == LXW_PREC_MIXED;
  return a;
}

int launch_any3(const lxw_solver3* s, double* Q, const Args3& a, cudaStream_t st, void** events) {
  if (s->kind == 1) return launch_step3t(s->deg, s->tm, s->dw, Q, a, st, s->opt.block_threads, events, 99);
  return launch_step3(s->deg, s->dm, s->dw, Q, a, st, s->opt.block_threads, events, 99);
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
    d->dt = a.dt_in > 0.0 ? a.dt_in : a.cfl * s->hmin / d->s;
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
  if (launch_any3(s, Q_dev, a, s->stream, nullptr)) return fail3(LXW_ERR_CUDA, "lxw3_step: launch failed");
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
    const int rc = launch_any3(s, Q_dev, a, s->cap_stream, nullptr);
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
  if (launch_any3(s, Q_dev, a, s->stream, (void**)s->ev)) return fail3(LXW_ERR_CUDA, "lxw3_profile_step: launch failed");
  LXW3_CUDA(cudaEventSynchronize(s->ev[5]));
  for (int k = 0; k < 5; ++k) LXW3_CUDA(cudaEventElapsedTime(&ms[k], s->ev[k], s->ev[k + 1]));
  return LXW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- tetrahedra
namespace {

// Jacobi polynomial P_n^(al, 0)(x), three-term recurrence in n
long double jacobi_host(int n, int al, long double x) {
  long double p0 = 1.0L;
  if (n == 0) return p0;
  long double p1 = 0.5L * ((al + 2) * x + al);
  for (int k = 2; k <= n; ++k) {
    const long double c = 2.0L * k + al;
    const long double p2 = ((c - 1) * (c * (c - 2) * x + (long double)al * al) * p1 - 2.0L * (k + al - 1) * (k - 1) * c * p0) /
                           (2.0L * k * (k + al) * (c - 2));
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// n-point Gauss rule on [0, 1] for the weight (1 - u)^al: the nodes are the
// zeros of P_n^(al, 0)(2u - 1), bracketed on a fine grid and bisected; each
// weight integrates the node's Lagrange polynomial times (1 - u)^al exactly
// (a Gauss-Legendre rule of n + 2 points).  Weights unnormalised.
void gauss_jacobi_host(int n, int al, double* u, double* w) {
  long double z[8];
  int found = 0;
  const int M = 4096;
  long double xa = -1.0L, fa = jacobi_host(n, al, xa);
  for (int q = 1; q <= M && found < n; ++q) {
    long double xb = -1.0L + 2.0L * q / M, fb = jacobi_host(n, al, xb);
    if (fb == 0.0L) {
      z[found++] = xb;   // a node on the grid (x = 0 for odd n and al = 0)
    } else if (fa != 0.0L && (fa < 0.0L) != (fb < 0.0L)) {
      long double lo = xa, hi = xb, flo = fa;
      for (int it = 0; it < 100; ++it) {
        const long double mid = 0.5L * (lo + hi), fm = jacobi_host(n, al, mid);
        if ((fm < 0.0L) == (flo < 0.0L)) { lo = mid; flo = fm; } else { hi = mid; }
      }
      z[found++] = 0.5L * (lo + hi);
    }
    xa = xb; fa = fb;
  }
  double g[10], gw[10];
  host_gauss_legendre(n + 2, g, gw);
  for (int j = 0; j < n; ++j) {
    long double acc = 0.0L;
    for (int q = 0; q < n + 2; ++q) {
      long double l = 1.0L;
      for (int a = 0; a < al; ++a) l *= 1.0L - g[q];
      for (int i = 0; i < n; ++i)
        if (i != j) l *= (g[q] - z[i]) / (z[j] - z[i]);
      acc += gw[q] * l;
    }
    u[j] = (double)(0.5L * (z[j] + 1.0L));
    w[j] = (double)acc;
  }
}

// Orthonormal basis on T0 (under (1/|T0|) Int): phi = L^-1 m, with m the
// monomials r^a s^b t^c in mode order and L L^T their Gram matrix, whose
// entries are 6 a! b! c! / (a + b + c + 3)! in closed form.  The rows of
// L^-1 are the Gram-Schmidt orthonormalisation of m in that order.
struct TetBasis {
  int deg = 0, ML = 0;
  std::vector<int> abc;
  long double C[k3MaxML][k3MaxML] = {};   // phi_l = sum_j C[l][j] m_j
  void init(int d) {
    deg = d; ML = modes3(d);
    exponents3(d, abc);
    auto fact = [](int n) { long double f = 1.0L; for (int k = 2; k <= n; ++k) f *= k; return f; };
    long double G[k3MaxML][k3MaxML], L[k3MaxML][k3MaxML] = {};
    for (int i = 0; i < ML; ++i)
      for (int j = 0; j < ML; ++j) {
        const int a = abc[3 * i] + abc[3 * j], b = abc[3 * i + 1] + abc[3 * j + 1], c = abc[3 * i + 2] + abc[3 * j + 2];
        G[i][j] = 6.0L * fact(a) * fact(b) * fact(c) / fact(a + b + c + 3);
      }
    for (int j = 0; j < ML; ++j) {   // Cholesky
      long double d2 = G[j][j];
      for (int k = 0; k < j; ++k) d2 -= L[j][k] * L[j][k];
      L[j][j] = sqrtl(d2);
      for (int i = j + 1; i < ML; ++i) {
        long double v = G[i][j];
        for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
        L[i][j] = v / L[j][j];
      }
    }
    for (int col = 0; col < ML; ++col)   // C = L^-1 by forward substitution
      for (int i = 0; i < ML; ++i) {
        long double v = (i == col) ? 1.0L : 0.0L;
        for (int k = 0; k < i; ++k) v -= L[i][k] * C[k][col];
        C[i][col] = v / L[i][i];
      }
  }
  void eval(const double r[3], double* phi, double* grad /* [3][ML] or null */) const {
    long double pw[3][4], dp[3][4];
    for (int ax = 0; ax < 3; ++ax) {
      pw[ax][0] = 1.0L; dp[ax][0] = 0.0L;
      for (int n = 1; n <= deg; ++n) { pw[ax][n] = pw[ax][n - 1] * r[ax]; dp[ax][n] = n * pw[ax][n - 1]; }
    }
    long double m[k3MaxML], g[3][k3MaxML];
    for (int j = 0; j < ML; ++j) {
      const int a = abc[3 * j], b = abc[3 * j + 1], c = abc[3 * j + 2];
      m[j] = pw[0][a] * pw[1][b] * pw[2][c];
      g[0][j] = dp[0][a] * pw[1][b] * pw[2][c];
      g[1][j] = pw[0][a] * dp[1][b] * pw[2][c];
      g[2][j] = pw[0][a] * pw[1][b] * dp[2][c];
    }
    for (int l = 0; l < ML; ++l) {
      long double v = 0.0L, x = 0.0L, y = 0.0L, z = 0.0L;
      for (int j = 0; j <= l; ++j) { v += C[l][j] * m[j]; x += C[l][j] * g[0][j]; y += C[l][j] * g[1][j]; z += C[l][j] * g[2][j]; }
      phi[l] = (double)v;
      if (grad) { grad[l] = (double)x; grad[ML + l] = (double)y; grad[2 * ML + l] = (double)z; }
    }
  }
};

// conical-product rule on T0 with n points per direction (exact to degree
// 2n - 1): r = u, s = v (1 - u), t = w (1 - u) (1 - v); weights sum to 1
void tet_rule_host(int n, std::vector<double>& pts, std::vector<double>& wts) {
  double ua[8], uw[8], va[8], vw[8], wa[8], ww[8];
  gauss_jacobi_host(n, 2, ua, uw);
  gauss_jacobi_host(n, 1, va, vw);
  gauss_jacobi_host(n, 0, wa, ww);
  pts.clear(); wts.clear();
  double tot = 0.0;
  for (int c = 0; c < n; ++c)
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        pts.insert(pts.end(), {ua[a], va[b] * (1.0 - ua[a]), wa[c] * (1.0 - ua[a]) * (1.0 - va[b])});
        wts.push_back(uw[a] * vw[b] * ww[c]);
        tot += wts.back();
      }
  for (double& x : wts) x /= tot;
}

const double kTRef[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// Tables of one degree: interior rule and basis, differentiation tables,
// the face tables fphi[k][perm][NF][ML], and the projection rule.
void make_tables3t(int deg, Tables3T& t, std::vector<double>& fphi, std::vector<double>& pj, std::vector<double>& jw,
                   std::vector<double>& jphi) {
  std::memset(&t, 0, sizeof(t));
  TetBasis B;
  B.init(deg);
  const int ML = B.ML, n = deg + 1;
  std::vector<double> pts, wts;
  tet_rule_host(n, pts, wts);
  const int NQ = (int)wts.size();
  std::vector<double> grad(3 * ML);
  for (int k = 0; k < NQ; ++k) {
    t.qw[k] = wts[k];
    B.eval(&pts[3 * k], t.phi[k], grad.data());
    for (int ax = 0; ax < 3; ++ax)
      for (int l = 0; l < ML; ++l) t.dref[ax][k][l] = grad[ax * ML + l];
  }
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
  // triangle rule: (a, b) = (u, v (1 - u)), weight (1 - u) in u
  double ua[8], uw[8], va[8], vw[8];
  gauss_jacobi_host(n, 1, ua, uw);
  gauss_jacobi_host(n, 0, va, vw);
  std::vector<double> fa, fb;
  double tot = 0.0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      fa.push_back(ua[i]); fb.push_back(va[j] * (1.0 - ua[i]));
      t.fw[j * n + i] = uw[i] * vw[j];
      tot += uw[i] * vw[j];
    }
  const int NF = n * n;
  for (int p = 0; p < NF; ++p) t.fw[p] /= tot;
  fphi.assign((size_t)4 * k3tPerms * NF * ML, 0.0);
  for (int k = 0; k < 4; ++k) {
    int o[3], c = 0;
    for (int v = 0; v < 4; ++v)
      if (v != k) o[c++] = v;
    for (int pm = 0; pm < k3tPerms; ++pm) {
      const int lv[3] = {o[kPerm[pm][0]], o[kPerm[pm][1]], o[kPerm[pm][2]]};
      for (int p = 0; p < NF; ++p) {
        const double lam[3] = {1.0 - fa[p] - fb[p], fa[p], fb[p]};
        double r[3];
        for (int d = 0; d < 3; ++d) r[d] = lam[0] * kTRef[lv[0]][d] + lam[1] * kTRef[lv[1]][d] + lam[2] * kTRef[lv[2]][d];
        B.eval(r, &fphi[((size_t)(k * k3tPerms + pm) * NF + p) * ML], nullptr);
      }
    }
  }
  for (int k = 0; k < NQ; ++k)
    for (int l = 0; l < ML; ++l) t.phimax[l] = std::max(t.phimax[l], std::fabs(t.phi[k][l]));
  for (size_t e = 0; e < fphi.size(); ++e) t.phimax[e % ML] = std::max(t.phimax[e % ML], std::fabs(fphi[e]));
  // projection rule: deg + 3 points per direction
  std::vector<double> jp, jwt;
  tet_rule_host(deg + 3, jp, jwt);
  pj = jp; jw = jwt;
  jphi.assign(jwt.size() * ML, 0.0);
  for (size_t p = 0; p < jwt.size(); ++p) B.eval(&jp[3 * p], &jphi[p * ML], nullptr);
}

}  // namespace

extern "C" {

lxw_status lxw3_solver_create_tets(int n_vertices, const double* xyz, int n_tets, const int* tets, const int* vid,
                                   const int* face_bc, int degree, const lxw_options* optp, void* stream,
                                   lxw_solver3** out) {
  const char* who = "lxw3_solver_create_tets";
  if (!out || !xyz || !tets || !vid) return fail3(LXW_ERR_ARG, std::string(who) + ": null argument");
  *out = nullptr;
  if (n_vertices < 4 || n_tets < 1) return fail3(LXW_ERR_ARG, std::string(who) + ": need >= 4 vertices and >= 1 cell");
  if (n_tets > (1 << 30)) return fail3(LXW_ERR_ARG, std::string(who) + ": more than 2^30 cells");
  if (degree < 1 || degree > 2) return fail3(LXW_ERR_ARG, std::string(who) + ": degree must be 1 or 2");
  lxw_options opt;
  if (lxw_status st = options3(optp, who, opt)) return st;
  const size_t N = (size_t)n_tets;
  // per-cell geometry
  std::vector<double> hgeo((size_t)k3tGeo * N), org(3 * N), jac(9 * N);
  for (size_t i = 0; i < N; ++i) {
    const int* v = tets + 4 * i;
    for (int a = 0; a < 4; ++a) {
      if (v[a] < 0 || v[a] >= n_vertices) return fail3(LXW_ERR_ARG, std::string(who) + ": vertex index out of range");
      for (int b = 0; b < a; ++b)
        if (vid[v[a]] == vid[v[b]]) return fail3(LXW_ERR_ARG, std::string(who) + ": a cell repeats a vertex id");
    }
    double J[9];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) J[3 * a + b] = xyz[3 * v[b + 1] + a] - xyz[3 * v[0] + a];
    const double c00 = J[4] * J[8] - J[5] * J[7], c01 = J[5] * J[6] - J[3] * J[8], c02 = J[3] * J[7] - J[4] * J[6];
    const double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
    if (!(det > 0.0)) return fail3(LXW_ERR_ARG, std::string(who) + ": cells must be positively oriented");
    // inverse: rows are d r_a / d x
    const double Ji[9] = {c00 / det, (J[2] * J[7] - J[1] * J[8]) / det, (J[1] * J[5] - J[2] * J[4]) / det,
                          c01 / det, (J[0] * J[8] - J[2] * J[6]) / det, (J[2] * J[3] - J[0] * J[5]) / det,
                          c02 / det, (J[1] * J[6] - J[0] * J[7]) / det, (J[0] * J[4] - J[1] * J[3]) / det};
    for (int e = 0; e < 9; ++e) { hgeo[e * N + i] = Ji[e]; jac[9 * i + e] = J[e]; }
    hgeo[9 * N + i] = det / 6.0;
    for (int d = 0; d < 3; ++d) org[3 * i + d] = xyz[3 * v[0] + d];
  }
  // faces: canonical vertex order (ascending id), its perm, matching by the sorted ids
  struct FaceRec { int a, b, c, cell, k; };
  std::vector<FaceRec> rec(4 * N);
  std::vector<int> code(N, 0), hnbr(4 * N);
  std::vector<int> canon(12 * N);
  for (size_t i = 0; i < N; ++i) {
    const int* v = tets + 4 * i;
    for (int k = 0; k < 4; ++k) {
      int o[3], c = 0;
      for (int a = 0; a < 4; ++a)
        if (a != k) o[c++] = a;
      int lv[3] = {o[0], o[1], o[2]};
      for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
          if (vid[v[lv[b]]] < vid[v[lv[a]]]) std::swap(lv[a], lv[b]);
      int pm = 0;
      while (!(o[kPerm[pm][0]] == lv[0] && o[kPerm[pm][1]] == lv[1] && o[kPerm[pm][2]] == lv[2])) ++pm;
      code[i] |= pm << (3 * k);
      for (int a = 0; a < 3; ++a) canon[12 * i + 3 * k + a] = lv[a];
      rec[4 * i + k] = {vid[v[lv[0]]], vid[v[lv[1]]], vid[v[lv[2]]], (int)i, k};
    }
  }
  std::sort(rec.begin(), rec.end(), [](const FaceRec& x, const FaceRec& y) {
    if (x.a != y.a) return x.a < y.a;
    if (x.b != y.b) return x.b < y.b;
    if (x.c != y.c) return x.c < y.c;
    return x.cell * 4 + x.k < y.cell * 4 + y.k;
  });
  // outward normal scaled by the area of face k of cell i, from its canonical vertices
  auto area_normal = [&](size_t i, int k, double an[3]) {
    const int* v = tets + 4 * i;
    const int* lv = &canon[12 * i + 3 * k];
    const double *pa = xyz + 3 * v[lv[0]], *pb = xyz + 3 * v[lv[1]], *pc = xyz + 3 * v[lv[2]], *po = xyz + 3 * v[k];
    const double e1[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
    const double e2[3] = {pc[0] - pa[0], pc[1] - pa[1], pc[2] - pa[2]};
    an[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);
    an[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
    an[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
    if (an[0] * (po[0] - pa[0]) + an[1] * (po[1] - pa[1]) + an[2] * (po[2] - pa[2]) > 0.0)
      for (int d = 0; d < 3; ++d) an[d] = -an[d];
  };
  auto put_normal = [&](size_t i, int k, const double an[3], double sg) {
    for (int d = 0; d < 3; ++d) hgeo[(size_t)(10 + 3 * k + d) * N + i] = sg * an[d];
    hgeo[(size_t)(22 + k) * N + i] = std::sqrt(an[0] * an[0] + an[1] * an[1] + an[2] * an[2]);
  };
  for (size_t r = 0; r < rec.size();) {
    size_t e = r + 1;
    while (e < rec.size() && rec[e].a == rec[r].a && rec[e].b == rec[r].b && rec[e].c == rec[r].c) ++e;
    if (e - r > 2) return fail3(LXW_ERR_ARG, std::string(who) + ": a face is shared by more than two cells");
    const FaceRec& f = rec[r];
    double an[3];
    area_normal(f.cell, f.k, an);   // the owner: the lower (cell, face)
    put_normal(f.cell, f.k, an, 1.0);
    if (e - r == 2) {
      const FaceRec& g = rec[r + 1];
      put_normal(g.cell, g.k, an, -1.0);
      hnbr[(size_t)f.k * N + f.cell] = g.cell;
      hnbr[(size_t)g.k * N + g.cell] = f.cell;
      code[f.cell] |= g.k << (12 + 2 * f.k);
      code[g.cell] |= f.k << (12 + 2 * g.k);
    } else {
      const int bc = face_bc ? face_bc[4 * (size_t)f.cell + f.k] : LXW_BC_TRANSPARENT;
      if (bc != LXW_BC_REFLECT && bc != LXW_BC_TRANSPARENT)
        return fail3(LXW_ERR_ARG, std::string(who) + ": an unmatched face must be reflective or transparent");
      hnbr[(size_t)f.k * N + f.cell] = -1 - bc;
    }
    r = e;
  }
  double hmin = 1e300;
  for (size_t i = 0; i < N; ++i) {
    double surf = 0.0;
    for (int k = 0; k < 4; ++k) surf += hgeo[(size_t)(22 + k) * N + i];
    hmin = std::min(hmin, 3.0 * hgeo[9 * N + i] / surf);
  }
  lxw_solver3* s = new (std::nothrow) lxw_solver3;
  if (!s) return fail3(LXW_ERR_NOMEM, std::string(who) + ": host allocation failed");
  s->kind = 1; s->E = 4;
  s->N = (int)N; s->deg = degree; s->ML = modes3(degree); s->NF = (degree + 1) * (degree + 1);
  s->opt = opt;
  s->stream = (cudaStream_t)stream;
  s->hmin = hmin;
  s->org.swap(org);
  s->jac.swap(jac);
  Tables3T t;
  std::vector<double> fphi, jw, jphi;
  make_tables3t(degree, t, fphi, s->pj, jw, jphi);
  s->NPJ = (int)jw.size();
  if (upload_tables3t(degree, t)) { delete s; return fail3(LXW_ERR_CUDA, std::string(who) + ": table upload failed"); }
  auto dalloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    s->allocs.push_back(p);
    return p;
  };
  double* dgeo = (double*)dalloc(sizeof(double) * hgeo.size());
  int* dnbr = (int*)dalloc(sizeof(int) * hnbr.size());
  int* dcode = (int*)dalloc(sizeof(int) * N);
  double* dfphi = (double*)dalloc(sizeof(double) * fphi.size());
  float* dfphif = (float*)dalloc(sizeof(float) * fphi.size());
  std::vector<float> fphif(fphi.begin(), fphi.end());
  s->dw.trace = (double*)dalloc(sizeof(double) * 4 * s->NF * 10 * N);
  s->dw.flux = (double*)dalloc(sizeof(double) * 40 * N);
  s->dw.prop = (double*)dalloc(sizeof(double) * 4 * N);
  s->dw.fbar = (double*)dalloc(sizeof(double) * 15 * N);
  s->dw.smax = (unsigned long long*)dalloc(sizeof(unsigned long long));
  s->dw.status = (unsigned int*)dalloc(sizeof(unsigned int));
  s->dw.diag = (Diag3Block*)dalloc(sizeof(Diag3Block));
  s->jw = (double*)dalloc(sizeof(double) * jw.size());
  s->jphi = (double*)dalloc(sizeof(double) * jphi.size());
  if (!dgeo || !dnbr || !dcode || !dfphi || !dfphif || !s->dw.trace || !s->dw.flux || !s->dw.prop || !s->dw.fbar || !s->dw.smax ||
      !s->dw.status || !s->dw.diag || !s->jw || !s->jphi) {
    delete s;
    return fail3(LXW_ERR_NOMEM, std::string(who) + ": device allocation failed");
  }
  cudaError_t e = cudaMemcpy(dgeo, hgeo.data(), sizeof(double) * hgeo.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dnbr, hnbr.data(), sizeof(int) * hnbr.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dcode, code.data(), sizeof(int) * N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dfphi, fphi.data(), sizeof(double) * fphi.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dfphif, fphif.data(), sizeof(float) * fphif.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->jw, jw.data(), sizeof(double) * jw.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->jphi, jphi.data(), sizeof(double) * jphi.size(), cudaMemcpyHostToDevice);
  for (int k = 0; k < 8 && e == cudaSuccess; ++k) e = cudaEventCreate(&s->ev[k]);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete s;
    return fail3(LXW_ERR_CUDA, std::string(who) + ": " + cudaGetErrorString(e));
  }
  s->tm.N = (int)N;
  s->tm.hmin = hmin;
  s->tm.geo = dgeo;
  s->tm.nbr = dnbr;
  s->tm.code = dcode;
  s->tm.fphi = dfphi;
  s->tm.fphif = dfphif;
  *out = s;
  return LXW_OK;
}

}  // extern "C"
