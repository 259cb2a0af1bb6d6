// lxw_host.cpp -- host side of the library: quadrature and modal basis
// tables, mesh connectivity and geometry, device memory of a solver, CUDA
// graph replay, and the extern "C" entry points declared in include/lxw.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "lxw_internal.h"
#include "lxw_internal3d.h"

namespace lxw {
void decode_diag(const double* raw, double out[9]);
size_t diag_bytes();
}  // namespace lxw

using namespace lxw;

namespace {

thread_local std::string g_err;

lxw_status fail(lxw_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

#define LXW_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(LXW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ------------------------------------------------------------- quadrature
// Gauss-Legendre nodes on [-1,1]: Newton iteration on P_n from Tricomi's
// asymptotic initial guesses, in long double; weights 2/((1-x^2) P_n'(x)^2).
// The lower half is computed and mirrored, so x[n-1-i] = -x[i] exactly.
void legendre_eval(int n, long double x, long double& p, long double& dp) {
  long double a = 1.0L, b = x;
  if (n == 0) { p = 1.0L; dp = 0.0L; return; }
  for (int k = 1; k < n; ++k) {
    long double c = ((2 * k + 1) * x * b - k * a) / (k + 1);
    a = b; b = c;
  }
  p = b;
  dp = n * (a - x * b) / (1.0L - x * x);
}

void gauss_legendre(int n, double* x, double* w) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n / 2 + n % 2; ++i) {
    long double th = pi * (4 * (i + 1) - 1) / (4 * n + 2);
    long double z = (1.0L - (n - 1.0L) / (8.0L * n * n * n)) * cosl(th);
    for (int it = 0; it < 50; ++it) {
      long double p, dp;
      legendre_eval(n, z, p, dp);
      long double step = p / dp;
      z -= step;
      if (fabsl(step) < 1e-30L) break;
    }
    long double p, dp;
    legendre_eval(n, z, p, dp);
    long double wi = 2.0L / ((1.0L - z * z) * dp * dp);
    x[i] = (double)(-z); x[n - 1 - i] = (double)z;
    w[i] = (double)wi; w[n - 1 - i] = (double)wi;
  }
  if (n % 2) x[n / 2] = 0.0;
}

// normalised Legendre value/derivative, (1/2) Int_{-1}^{1} L_n^2 = 1.  The
// derivative follows P'_{k+1} = P'_{k-1} + (2k+1) P_k, which has no
// division and so holds at the edge points x = +-1 of the reference square.
void legendre_norm(int n, double x, double& v, double& d) {
  long double p0 = 1.0L, p1 = x, d0 = 0.0L, d1 = 1.0L;
  long double p = 1.0L, dp = 0.0L;
  if (n == 1) { p = p1; dp = d1; }
  for (int k = 1; k < n; ++k) {
    long double p2 = ((2 * k + 1) * (long double)x * p1 - k * p0) / (k + 1);
    long double d2 = d0 + (2 * k + 1) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
    p = p2; dp = d2;
  }
  long double s = sqrtl(2.0L * n + 1.0L);
  v = (double)(s * p);
  d = (double)(s * dp);
}

// interior rule with n points per direction, weights summing to 1
int interior_rule(int kind, int n, double* xi, double* eta, double* w) {
  double g[8], gw[8];
  gauss_legendre(n, g, gw);
  int c = 0;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b, ++c) {
      if (kind == LXW_KIND_QUAD) {
        xi[c] = g[a]; eta[c] = g[b]; w[c] = 0.25 * gw[a] * gw[b];
      } else {
        // collapsed coordinates x = u, y = v (1 - u) on the reference triangle
        double u = 0.5 + 0.5 * g[a], v = 0.5 + 0.5 * g[b];
        xi[c] = u; eta[c] = v * (1.0 - u);
        w[c] = 0.5 * gw[a] * gw[b] * (1.0 - u);
      }
    }
  return c;
}

// ------------------------------------------------------------ modal basis
// Quadrilateral: products of normalised Legendre polynomials, ordered by
// total degree: (0,0),(1,0),(0,1),(1,1),(2,0),(0,2),(3,0),(2,1),(1,2),(0,3).
// Triangle: the monomials 1,x,y,x^2,xy,y^2,x^3,x^2y,xy^2,y^3 orthonormalised
// in that order under (1/|T0|) Int_T0 (the Cholesky factor of their exact
// Gram matrix, 2 a! b!/(a+b+2)!), computed in long double.
const int kQA[10] = {0, 1, 0, 1, 2, 0, 3, 2, 1, 0};
const int kQB[10] = {0, 0, 1, 1, 0, 2, 0, 1, 2, 3};
const int kMA[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
const int kMB[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};

struct TriBasis { double c[kMaxML][kMaxML]; };  // phi_l = sum_j c[l][j] m_j

TriBasis triangle_basis(int ML) {
  long double G[kMaxML][kMaxML], L[kMaxML][kMaxML] = {};
  auto fac = [](int n) { long double f = 1.0L; for (int k = 2; k <= n; ++k) f *= k; return f; };
  for (int a = 0; a < ML; ++a)
    for (int b = 0; b < ML; ++b) {
      int p = kMA[a] + kMA[b], q = kMB[a] + kMB[b];
      G[a][b] = 2.0L * fac(p) * fac(q) / fac(p + q + 2);
    }
  // G = L L^T
  for (int r = 0; r < ML; ++r)
    for (int col = 0; col <= r; ++col) {
      long double s = G[r][col];
      for (int k = 0; k < col; ++k) s -= L[r][k] * L[col][k];
      L[r][col] = (r == col) ? sqrtl(s) : s / L[col][col];
    }
  // rows of L^{-1} are the coefficients of the orthonormal polynomials
  long double Li[kMaxML][kMaxML] = {};
  for (int col = 0; col < ML; ++col) {
    for (int r = 0; r < ML; ++r) {
      long double s = (r == col) ? 1.0L : 0.0L;
      for (int k = 0; k < r; ++k) s -= L[r][k] * Li[k][col];
      Li[r][col] = s / L[r][r];
    }
  }
  TriBasis tb{};
  for (int l = 0; l < ML; ++l)
    for (int j = 0; j < ML; ++j) tb.c[l][j] = (double)Li[l][j];
  return tb;
}

void basis_at(int kind, int ML, const TriBasis& tb, double x, double y, double* phi, double* dx, double* dy) {
  for (int l = 0; l < ML; ++l) {
    if (kind == LXW_KIND_QUAD) {
      double a, da, b, db;
      legendre_norm(kQA[l], x, a, da);
      legendre_norm(kQB[l], y, b, db);
      phi[l] = a * b; if (dx) dx[l] = da * b; if (dy) dy[l] = a * db;
    } else {
      double v = 0.0, vx = 0.0, vy = 0.0;
      for (int j = 0; j < ML; ++j) {
        int pa = kMA[j], pb = kMB[j];
        double xa = 1.0, yb = 1.0, xa1 = 0.0, yb1 = 0.0;
        for (int k = 0; k < pa; ++k) { xa1 = (k == pa - 1) ? xa * pa : xa1; xa *= x; }
        for (int k = 0; k < pb; ++k) { yb1 = (k == pb - 1) ? yb * pb : yb1; yb *= y; }
        v += tb.c[l][j] * xa * yb;
        vx += tb.c[l][j] * xa1 * yb;
        vy += tb.c[l][j] * xa * yb1;
      }
      phi[l] = v; if (dx) dx[l] = vx; if (dy) dy[l] = vy;
    }
  }
}

const double kQuadV[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
const double kTriV[3][2] = {{0, 0}, {1, 0}, {0, 1}};

void build_tables(int kind, int deg, Tables& t, ProjTables& pt) {
  std::memset(&t, 0, sizeof(t));
  std::memset(&pt, 0, sizeof(pt));
  const int ML = (deg + 1) * (deg + 2) / 2, n = deg + 1;
  const int E = kind == LXW_KIND_QUAD ? 4 : 3;
  TriBasis tb = kind == LXW_KIND_TRI ? triangle_basis(ML) : TriBasis{};
  t.ML = ML; t.E = E; t.MQ = n;
  double xi[kMaxPts], eta[kMaxPts], w[kMaxQ];
  t.NQ = interior_rule(kind, n, xi, eta, w);
  for (int k = 0; k < t.NQ; ++k) t.w[k] = w[k];
  double g[8], gw[8];
  gauss_legendre(n, g, gw);
  for (int p = 0; p < n; ++p) t.ew[p] = gw[p];
  const double(*V)[2] = kind == LXW_KIND_QUAD ? kQuadV : kTriV;
  for (int k = 0; k < E; ++k)
    for (int p = 0; p < n; ++p) {
      double s = 0.5 * (g[p] + 1.0);
      int idx = t.NQ + k * n + p;
      xi[idx] = V[k][0] + s * (V[(k + 1) % E][0] - V[k][0]);
      eta[idx] = V[k][1] + s * (V[(k + 1) % E][1] - V[k][1]);
    }
  t.NPT = t.NQ + E * n;
  for (int p = 0; p < t.NPT; ++p) basis_at(kind, ML, tb, xi[p], eta[p], t.phi[p], t.dxi[p], t.deta[p]);
  // projection rule: deg + 3 points per direction
  double pxi[kMaxProj], peta[kMaxProj], pw[kMaxProj];
  pt.ML = ML;
  pt.NPJ = interior_rule(kind, deg + 3, pxi, peta, pw);
  t.NPJ = pt.NPJ;
  for (int p = 0; p < pt.NPJ; ++p) {
    pt.w[p] = pw[p];
    basis_at(kind, ML, tb, pxi[p], peta[p], pt.phi[p], nullptr, nullptr);
  }
}

void projection_reference_points(int kind, int deg, std::vector<double>& xi, std::vector<double>& eta) {
  double a[kMaxProj], b[kMaxProj], w[kMaxProj];
  int n = interior_rule(kind, deg + 3, a, b, w);
  xi.assign(a, a + n); eta.assign(b, b + n);
}

}  // namespace

void lxw::set_last_error(const char* msg) { g_err = msg; }
void lxw::host_gauss_legendre(int n, double* x, double* w) { gauss_legendre(n, x, w); }
void lxw::host_legendre_norm(int n, double x, double& v, double& d) { legendre_norm(n, x, v, d); }

void lxw::make_deriv_tables(const Tables& t, DerivTables& d) {
  std::memset(&d, 0, sizeof(d));
  double D[2][kMaxML][kMaxML] = {};
  for (int m = 0; m < t.ML; ++m)
    for (int l = 0; l < t.ML; ++l)
      for (int k = 0; k < t.NQ; ++k) {
        D[0][m][l] += t.w[k] * t.dxi[k][m] * t.phi[k][l];
        D[1][m][l] += t.w[k] * t.deta[k][m] * t.phi[k][l];
      }
  for (int c = 0; c < 2; ++c)
    for (int k = 0; k < t.NQ; ++k)
      for (int l = 0; l < t.ML; ++l) {
        double acc = 0.0;
        for (int m = 0; m < t.ML; ++m) acc += t.phi[k][m] * D[c][m][l];
        d.W[c][k][l] = t.w[k] * acc;
      }
}

void lxw::make_tables(int kind, int deg, Tables& t) {
  ProjTables pt;
  build_tables(kind, deg, t, pt);
}

// ------------------------------------------------------------------ mesh
struct lxw_mesh {
  int kind, N, E;
  std::vector<double> vx;   // [N][E][2]
  std::vector<int> nbr;     // [N][E]: neighbour or -1 - bc
  std::vector<int> nbk;     // [N][E]
};

struct lxw_solver {
  int kind, deg, N, E, ML;
  lxw_options opt;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  Tables tab;
  ProjTables ptab;
  DevMesh dm{};
  DevWork dw{};
  DevWorkMx dwm{};               // mixed form workspace
  bool mixed = false;
  std::vector<int> pstart;       // problem element ranges [nprob + 1]
  std::vector<double> hmin_p;    // per problem
  int4* d_tiles = nullptr;       // work list (owned through allocs)
  GateWeights* gate_buf = nullptr;  // gate weights (owned), allocated by the first lxw_solver_set_mlp
  const GateWeights* mlp_w = nullptr;  // gate_buf while a network is attached, else null
  double qin[4] = {0.0, 0.0, 0.0, 0.0};  // conserved state of LXW_BC_INFLOW faces
  int gate_per_sm[2] = {1, 1};         // resident gate CTAs per SM of each variant (queried when a network is attached)
  float mlp_tau = 0.0f;
  long long gate_wait_test = 0;      // test aid of the gate's bounded waits (lxw_solver_set_gate_wait_test)
  int tiles_cap = 0;
  int sms = 0;
  std::vector<void*> allocs;
  double* Qdev = nullptr;        // FP64 staging buffer of lxw_run_host
  double* Sdev = nullptr;        // packed state of lxw_run_host (mixed form)
  double* host_diag = nullptr;   // pinned
  double* tclock = nullptr;      // [nprob][4] clocks of lxw_run_to (device)
  double* host_clock = nullptr;  // pinned copy of tclock
  cudaGraphExec_t tgraph = nullptr;   // one timed step (lxw_run_to)
  double* tgraph_Q = nullptr;
  double tgraph_cfl = 0.0, tgraph_tend = 0.0;
  std::vector<double> xproj;     // [N][NPJ][2]
  cudaGraphExec_t graph = nullptr;
  double* graph_Q = nullptr;
  double graph_cfl = 0.0;
  double last_dt_in = 0.0, last_cfl = 0.0;
  void* events[8] = {};          // cudaEvent_t of lxw_profile_step
  cudaGraphExec_t pgraph = nullptr;   // one step with event nodes between the kernels
  double* pgraph_Q = nullptr;
  double pgraph_cfl = 0.0;
  ~lxw_solver() {
    if (graph) cudaGraphExecDestroy(graph);
    if (tgraph) cudaGraphExecDestroy(tgraph);
    if (host_clock) cudaFreeHost(host_clock);
    if (pgraph) cudaGraphExecDestroy(pgraph);
    for (void* e : events) if (e) cudaEventDestroy((cudaEvent_t)e);
    for (void* p : allocs) cudaFree(p);
    if (host_diag) cudaFreeHost(host_diag);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

extern "C" {

const char* lxw_last_error(void) { return g_err.c_str(); }

lxw_status lxw_options_default(lxw_options* opt) {
  if (!opt) return fail(LXW_ERR_ARG, "lxw_options_default: null");
  std::memset(opt, 0, sizeof(*opt));
  opt->gamma = 1.4;
  opt->eps0 = 1e-12;
  opt->alpha0 = 500.0;
  opt->shock_limiter = 1;
  opt->precision = LXW_PREC_FP64;
  opt->block_threads = 128;
  opt->ck_order = 3;
  return LXW_OK;
}

lxw_status lxw_mesh_cartesian_masked(int nx, int ny, double x0, double x1, double y0, double y1, const int bc[4],
                                     const unsigned char* mask, int mask_bc, lxw_mesh** out) {
  if (!out || !bc) return fail(LXW_ERR_ARG, "lxw_mesh_cartesian: null argument");
  if (nx < 1 || ny < 1 || !(x1 > x0) || !(y1 > y0)) return fail(LXW_ERR_ARG, "lxw_mesh_cartesian: bad size or box");
  for (int k = 0; k < 4; ++k)
    if (bc[k] < LXW_BC_PERIODIC || bc[k] > LXW_BC_INFLOW) return fail(LXW_ERR_ARG, "lxw_mesh_cartesian: bad boundary code");
  if (mask_bc < LXW_BC_REFLECT || mask_bc > LXW_BC_INFLOW)
    return fail(LXW_ERR_ARG, "lxw_mesh_cartesian_masked: mask_bc must be REFLECT, TRANSPARENT or INFLOW");
  if ((bc[0] == LXW_BC_PERIODIC) != (bc[1] == LXW_BC_PERIODIC) || (bc[2] == LXW_BC_PERIODIC) != (bc[3] == LXW_BC_PERIODIC))
    return fail(LXW_ERR_ARG, "lxw_mesh_cartesian: periodic sides must be paired");
  // compact ids of the kept cells, row order
  std::vector<int> id((size_t)nx * ny);
  int N = 0;
  for (size_t c = 0; c < id.size(); ++c) id[c] = (!mask || mask[c]) ? N++ : -1;
  if (N < 1) return fail(LXW_ERR_ARG, "lxw_mesh_cartesian_masked: the mask keeps no cell");
  lxw_mesh* m = new (std::nothrow) lxw_mesh;
  if (!m) return fail(LXW_ERR_NOMEM, "lxw_mesh_cartesian: out of memory");
  m->kind = LXW_KIND_QUAD; m->N = N; m->E = 4;
  m->vx.resize((size_t)N * 8); m->nbr.resize((size_t)N * 4); m->nbk.resize((size_t)N * 4);
  std::vector<double> X(nx + 1), Y(ny + 1);
  for (int a = 0; a <= nx; ++a) X[a] = x0 + (x1 - x0) * a / nx;
  for (int b = 0; b <= ny; ++b) Y[b] = y0 + (y1 - y0) * b / ny;
  // local edges counter-clockwise from the lower-left vertex: bottom, right, top, left
  const int side_bc[4] = {bc[2], bc[1], bc[3], bc[0]};
  const int opposite[4] = {2, 3, 0, 1};
  for (int iy = 0; iy < ny; ++iy)
    for (int ix = 0; ix < nx; ++ix) {
      const int e = id[(size_t)iy * nx + ix];
      if (e < 0) continue;
      double* v = &m->vx[(size_t)e * 8];
      v[0] = X[ix]; v[1] = Y[iy]; v[2] = X[ix + 1]; v[3] = Y[iy]; v[4] = X[ix + 1]; v[5] = Y[iy + 1]; v[6] = X[ix]; v[7] = Y[iy + 1];
      int jx[4] = {ix, ix + 1, ix, ix - 1}, jy[4] = {iy - 1, iy, iy + 1, iy};
      for (int k = 0; k < 4; ++k) {
        int a = jx[k], b = jy[k];
        bool inside = a >= 0 && a < nx && b >= 0 && b < ny;
        if (!inside && side_bc[k] == LXW_BC_PERIODIC) { a = (a + nx) % nx; b = (b + ny) % ny; inside = true; }
        const int j = inside ? id[(size_t)b * nx + a] : -1;
        m->nbr[(size_t)e * 4 + k] = j >= 0 ? j : -1 - (inside ? mask_bc : side_bc[k]);
        m->nbk[(size_t)e * 4 + k] = j >= 0 ? opposite[k] : -1;
      }
    }
  *out = m;
  return LXW_OK;
}

lxw_status lxw_mesh_cartesian(int nx, int ny, double x0, double x1, double y0, double y1, const int bc[4],
                              lxw_mesh** out) {
  return lxw_mesh_cartesian_masked(nx, ny, x0, x1, y0, y1, bc, nullptr, LXW_BC_REFLECT, out);
}

lxw_status lxw_mesh_triangles(int nv, const double* xy, int nt, const int* tv, const int* ebc, lxw_mesh** out) {
  if (!out || !xy || !tv || nv < 3 || nt < 1) return fail(LXW_ERR_ARG, "lxw_mesh_triangles: bad argument");
  lxw_mesh* m = new (std::nothrow) lxw_mesh;
  if (!m) return fail(LXW_ERR_NOMEM, "lxw_mesh_triangles: out of memory");
  m->kind = LXW_KIND_TRI; m->N = nt; m->E = 3;
  m->vx.resize((size_t)nt * 6); m->nbr.assign((size_t)nt * 3, 0); m->nbk.assign((size_t)nt * 3, -1);
  std::unordered_map<uint64_t, int> open;   // undirected edge -> first (element*3 + k)
  open.reserve((size_t)nt * 2);
  for (int e = 0; e < nt; ++e) {
    for (int k = 0; k < 3; ++k) {
      int a = tv[3 * e + k];
      if (a < 0 || a >= nv) { delete m; return fail(LXW_ERR_BOUNDS, "lxw_mesh_triangles: vertex id out of range"); }
      m->vx[(size_t)e * 6 + 2 * k] = xy[2 * a];
      m->vx[(size_t)e * 6 + 2 * k + 1] = xy[2 * a + 1];
    }
    const double* v = &m->vx[(size_t)e * 6];
    double det = (v[2] - v[0]) * (v[5] - v[1]) - (v[4] - v[0]) * (v[3] - v[1]);
    if (!(det > 0.0)) { delete m; return fail(LXW_ERR_ARG, "lxw_mesh_triangles: triangle " + std::to_string(e) + " is not counter-clockwise"); }
    for (int k = 0; k < 3; ++k) {
      uint32_t a = (uint32_t)tv[3 * e + k], b = (uint32_t)tv[3 * e + (k + 1) % 3];
      uint64_t key = a < b ? ((uint64_t)a << 32 | b) : ((uint64_t)b << 32 | a);
      auto it = open.find(key);
      if (it == open.end()) {
        open.emplace(key, e * 3 + k);
      } else {
        int o = it->second;
        if (o < 0) { delete m; return fail(LXW_ERR_ARG, "lxw_mesh_triangles: edge shared by more than two triangles"); }
        int oe = o / 3, ok = o % 3;
        m->nbr[(size_t)e * 3 + k] = oe; m->nbk[(size_t)e * 3 + k] = ok;
        m->nbr[(size_t)oe * 3 + ok] = e; m->nbk[(size_t)oe * 3 + ok] = k;
        it->second = -1;
      }
    }
  }
  for (auto& kv : open)
    if (kv.second >= 0) {
      int e = kv.second / 3, k = kv.second % 3;
      int code = ebc ? ebc[kv.second] : LXW_BC_TRANSPARENT;
      if (code < LXW_BC_REFLECT || code > LXW_BC_INFLOW) { delete m; return fail(LXW_ERR_ARG, "lxw_mesh_triangles: boundary edges need a reflective, transparent or inflow code"); }
      m->nbr[(size_t)e * 3 + k] = -1 - code;
      m->nbk[(size_t)e * 3 + k] = -1;
    }
  *out = m;
  return LXW_OK;
}

void lxw_mesh_destroy(lxw_mesh* m) { delete m; }
int lxw_mesh_num_elements(const lxw_mesh* m) { return m ? m->N : 0; }

static lxw_status build_tiles(lxw_solver* s);

static lxw_status create_impl(const lxw_mesh* mesh, const std::vector<int>& pstart, int degree,
                              const lxw_options* optp, void* stream, lxw_solver** out) {
  if (!mesh || !out) return fail(LXW_ERR_ARG, "lxw_solver_create: null argument");
  if (degree != 2 && degree != 3) return fail(LXW_ERR_ARG, "lxw_solver_create: degree must be 2 or 3");
  lxw_options opt;
  if (optp) opt = *optp; else lxw_options_default(&opt);
  if (!(opt.gamma > 1.0)) return fail(LXW_ERR_ARG, "lxw_solver_create: gamma must exceed 1");
  if (opt.precision != LXW_PREC_FP64 && opt.precision != LXW_PREC_MIXED)
    return fail(LXW_ERR_ARG, "lxw_solver_create: unsupported precision");
  if (opt.block_threads <= 0) opt.block_threads = 128;
  if (opt.block_threads % 32 || opt.block_threads > 128)
    return fail(LXW_ERR_ARG, "lxw_solver_create: block_threads must be a multiple of 32, at most 128");
  if (opt.ctas_per_sm < 0 || opt.ctas_per_sm > 32) return fail(LXW_ERR_ARG, "lxw_solver_create: ctas_per_sm must be in [0, 32]");
  if (opt.high_occupancy != 0 && opt.high_occupancy != 1)
    return fail(LXW_ERR_ARG, "lxw_solver_create: high_occupancy must be 0 or 1");
  if (opt.moment_exact != 0 && opt.moment_exact != 1)
    return fail(LXW_ERR_ARG, "lxw_solver_create: moment_exact must be 0 or 1");
  if (opt.llf_global != 0 && opt.llf_global != 1)
    return fail(LXW_ERR_ARG, "lxw_solver_create: llf_global must be 0 or 1");
  if (opt.gate_scan != 0 && opt.gate_scan != 1)
    return fail(LXW_ERR_ARG, "lxw_solver_create: gate_scan must be 0 or 1");
  if (opt.ck_order == 0) opt.ck_order = 3;
  if (opt.ck_order != 3 && opt.ck_order != 4)
    return fail(LXW_ERR_ARG, "lxw_solver_create: ck_order must be 3 or 4");
  lxw_solver* s = new (std::nothrow) lxw_solver;
  if (!s) return fail(LXW_ERR_NOMEM, "lxw_solver_create: out of memory");
  s->kind = mesh->kind; s->deg = degree; s->N = mesh->N; s->E = mesh->E; s->opt = opt;
  s->stream = (cudaStream_t)stream;
  build_tables(mesh->kind, degree, s->tab, s->ptab);
  s->ML = s->tab.ML;
  const int N = s->N, E = s->E, MQ = s->tab.MQ;

  // geometry (affine map of the reference element) on the host
  std::vector<double> area(N), jinv((size_t)4 * N), nrm((size_t)E * 2 * N), sdx(N);
  std::vector<int> nbr((size_t)E * N), nbk((size_t)E * N);
  double hmin = 1e300;
  const int nprob = (int)pstart.size() - 1;
  s->pstart = pstart;
  s->hmin_p.assign(nprob, 1e300);
  s->xproj.resize((size_t)N * s->ptab.NPJ * 2);
  std::vector<double> pxi, peta;
  projection_reference_points(mesh->kind, degree, pxi, peta);
  for (int e = 0; e < N; ++e) {
    const double* v = &mesh->vx[(size_t)e * E * 2];
    double o[2], J[4];
    if (mesh->kind == LXW_KIND_QUAD) {
      // x = centre + diag(hx/2, hy/2) xi on [-1,1]^2
      o[0] = 0.5 * (v[0] + v[2]); o[1] = 0.5 * (v[1] + v[7]);
      J[0] = 0.5 * (v[2] - v[0]); J[1] = 0.0; J[2] = 0.0; J[3] = 0.5 * (v[7] - v[1]);
    } else {
      o[0] = v[0]; o[1] = v[1];
      J[0] = v[2] - v[0]; J[1] = v[4] - v[0]; J[2] = v[3] - v[1]; J[3] = v[5] - v[1];
    }
    const double det = J[0] * J[3] - J[1] * J[2];
    jinv[e] = J[3] / det; jinv[N + e] = -J[1] / det; jinv[2 * (size_t)N + e] = -J[2] / det; jinv[3 * (size_t)N + e] = J[0] / det;
    area[e] = (mesh->kind == LXW_KIND_QUAD ? 4.0 : 0.5) * det;
    double P = 0.0;
    for (int k = 0; k < E; ++k) {
      const int k1 = (k + 1) % E;
      const double nx = v[2 * k1 + 1] - v[2 * k + 1], ny = -(v[2 * k1] - v[2 * k]);
      nrm[(size_t)(2 * k) * N + e] = nx; nrm[(size_t)(2 * k + 1) * N + e] = ny;
      P += std::sqrt(nx * nx + ny * ny);
      nbr[(size_t)k * N + e] = mesh->nbr[(size_t)e * E + k];
      nbk[(size_t)k * N + e] = mesh->nbk[(size_t)e * E + k];
    }
    hmin = std::fmin(hmin, 2.0 * area[e] / P);
    {
      int pb = 0;
      while (pb + 1 < nprob && e >= pstart[pb + 1]) ++pb;
      s->hmin_p[pb] = std::fmin(s->hmin_p[pb], 2.0 * area[e] / P);
    }
    sdx[e] = mesh->kind == LXW_KIND_QUAD ? 2.0 * J[0] : std::sqrt(2.0 * area[e]);
    for (int p = 0; p < s->ptab.NPJ; ++p) {
      s->xproj[((size_t)e * s->ptab.NPJ + p) * 2] = o[0] + J[0] * pxi[p] + J[1] * peta[p];
      s->xproj[((size_t)e * s->ptab.NPJ + p) * 2 + 1] = o[1] + J[2] * pxi[p] + J[3] * peta[p];
    }
  }
  auto dalloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    s->allocs.push_back(p);
    return p;
  };
  double* d_area = (double*)dalloc(sizeof(double) * N);
  double* d_jinv = (double*)dalloc(sizeof(double) * 4 * N);
  double* d_nrm = (double*)dalloc(sizeof(double) * E * 2 * N);
  double* d_sdx = (double*)dalloc(sizeof(double) * N);
  int* d_nbr = (int*)dalloc(sizeof(int) * E * N);
  int* d_nbk = (int*)dalloc(sizeof(int) * E * N);
  s->dw.trace = (double*)dalloc(sizeof(double) * (size_t)E * MQ * 8 * N);
  s->dw.flux = (double*)dalloc(sizeof(double) * (size_t)E * 8 * N);
  s->dw.prop = (double*)dalloc(sizeof(double) * (size_t)E * N);
  s->dw.smax = (unsigned long long*)dalloc(sizeof(unsigned long long) * nprob);
  s->dw.status = (unsigned int*)dalloc(sizeof(unsigned int));
  s->dw.diag = (double*)dalloc(sizeof(DiagBlock) > diag_bytes() ? sizeof(DiagBlock) : diag_bytes());
  s->tclock = (double*)dalloc(sizeof(double) * 4 * nprob);
  s->Qdev = (double*)dalloc(sizeof(double) * (size_t)N * 4 * s->ML);
  s->mixed = opt.precision == LXW_PREC_MIXED;
  if (s->mixed) {
    // the FP32 traces / f^LxW fit in the FP64 buffers
    s->dwm.trace = reinterpret_cast<float*>(s->dw.trace);
    s->dwm.fw = reinterpret_cast<float*>(s->dw.flux);
    s->dwm.prop = reinterpret_cast<float*>(s->dw.prop);
    s->dwm.avg_new = (double*)dalloc(sizeof(double) * 4 * (size_t)N);
    s->dwm.avgn32 = (float*)dalloc(sizeof(float) * 4 * (size_t)N);
    s->dwm.done = (unsigned int*)dalloc(sizeof(unsigned int));
    s->dwm.gate_list = (int*)dalloc(sizeof(int) * (size_t)N);
    s->dwm.gate_count = (unsigned int*)dalloc(sizeof(unsigned int));
    s->dwm.scal = (ScalMx*)dalloc(sizeof(ScalMx) * nprob);
    s->dwm.smax = s->dw.smax; s->dwm.status = s->dw.status; s->dwm.diag = s->dw.diag;
    s->Sdev = (double*)dalloc(lxw_state_bytes(s));
    float* j32 = (float*)dalloc(sizeof(float) * 4 * (size_t)N);
    float* n32 = (float*)dalloc(sizeof(float) * (size_t)E * 2 * N);
    float* s32 = (float*)dalloc(sizeof(float) * (size_t)N);
    float* ia32 = (float*)dalloc(sizeof(float) * (size_t)N);
    double* ia64 = (double*)dalloc(sizeof(double) * (size_t)N);
    if (!s->dwm.avg_new || !s->dwm.avgn32 || !s->dwm.done ||
        cudaMemset(s->dwm.done, 0, sizeof(unsigned int)) != cudaSuccess || !s->dwm.gate_list || !s->dwm.gate_count ||
        cudaMemset(s->dwm.gate_count, 0, sizeof(unsigned int)) != cudaSuccess || !s->dwm.scal || !s->Sdev || !j32 ||
        !n32 || !s32 || !ia32 || !ia64) {
      delete s;
      return fail(LXW_ERR_NOMEM, "lxw_solver_create: device allocation failed");
    }
    std::vector<float> hj(jinv.begin(), jinv.end()), hn(nrm.begin(), nrm.end()), hs(sdx.begin(), sdx.end());
    std::vector<float> hia(N);
    std::vector<double> hia64(N);
    for (int e = 0; e < N; ++e) { hia64[e] = 1.0 / area[e]; hia[e] = (float)hia64[e]; }
    if (cudaMemcpy(j32, hj.data(), sizeof(float) * hj.size(), cudaMemcpyHostToDevice) ||
        cudaMemcpy(n32, hn.data(), sizeof(float) * hn.size(), cudaMemcpyHostToDevice) ||
        cudaMemcpy(s32, hs.data(), sizeof(float) * hs.size(), cudaMemcpyHostToDevice) ||
        cudaMemcpy(ia32, hia.data(), sizeof(float) * N, cudaMemcpyHostToDevice) ||
        cudaMemcpy(ia64, hia64.data(), sizeof(double) * N, cudaMemcpyHostToDevice)) {
      delete s;
      return fail(LXW_ERR_CUDA, "lxw_solver_create: upload failed");
    }
    s->dm.jinv32 = j32; s->dm.nrm32 = n32; s->dm.sdx32 = s32; s->dm.inva32 = ia32; s->dm.inva = ia64;
  }
  if (!d_area || !d_jinv || !d_nrm || !d_sdx || !d_nbr || !d_nbk || !s->dw.trace || !s->dw.flux || !s->dw.prop ||
      !s->dw.smax || !s->dw.status || !s->dw.diag || !s->Qdev || !s->tclock ||
      cudaMemset(s->dw.smax, 0, sizeof(unsigned long long) * nprob) != cudaSuccess ||
      cudaMemset(s->dw.status, 0, sizeof(unsigned int)) != cudaSuccess) {
    delete s;
    return fail(LXW_ERR_NOMEM, "lxw_solver_create: device allocation failed");
  }
  if (cudaMallocHost(&s->host_diag, 64 * sizeof(double)) != cudaSuccess) {
    s->host_diag = nullptr; delete s;
    return fail(LXW_ERR_NOMEM, "lxw_solver_create: pinned allocation failed");
  }
  if (cudaMallocHost(&s->host_clock, 4 * sizeof(double) * nprob) != cudaSuccess) {
    s->host_clock = nullptr; delete s;
    return fail(LXW_ERR_NOMEM, "lxw_solver_create: pinned allocation failed");
  }
  for (auto& e : s->events) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) { delete s; return fail(LXW_ERR_CUDA, "lxw_solver_create: event creation failed"); }
    e = ev;
  }
  if (cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    s->cap_stream = nullptr; delete s;
    return fail(LXW_ERR_CUDA, "lxw_solver_create: stream creation failed");
  }
  cudaError_t e1 = cudaMemcpy(d_area, area.data(), sizeof(double) * N, cudaMemcpyHostToDevice);
  cudaError_t e2 = cudaMemcpy(d_jinv, jinv.data(), sizeof(double) * 4 * N, cudaMemcpyHostToDevice);
  cudaError_t e3 = cudaMemcpy(d_nrm, nrm.data(), sizeof(double) * E * 2 * N, cudaMemcpyHostToDevice);
  cudaError_t e4 = cudaMemcpy(d_sdx, sdx.data(), sizeof(double) * N, cudaMemcpyHostToDevice);
  cudaError_t e5 = cudaMemcpy(d_nbr, nbr.data(), sizeof(int) * E * N, cudaMemcpyHostToDevice);
  cudaError_t e6 = cudaMemcpy(d_nbk, nbk.data(), sizeof(int) * E * N, cudaMemcpyHostToDevice);
  if (e1 || e2 || e3 || e4 || e5 || e6 || upload_tables(s->kind, degree, s->tab) ||
      (s->mixed && upload_tables_mx(s->kind, degree, s->tab))) {
    delete s;
    return fail(LXW_ERR_CUDA, "lxw_solver_create: upload failed");
  }
  s->dm.N = N; s->dm.E = E; s->dm.area = d_area; s->dm.jinv = d_jinv; s->dm.nrm = d_nrm; s->dm.sdx = d_sdx;
  // (FP32 geometry copies of the mixed form were set above)
  s->dm.nbr = d_nbr; s->dm.nbk = d_nbk; s->dm.hmin = s->hmin_p[0];
  s->dm.nprob = nprob;
  double* d_hp = (double*)dalloc(sizeof(double) * nprob);
  if (!d_hp || cudaMemcpy(d_hp, s->hmin_p.data(), sizeof(double) * nprob, cudaMemcpyHostToDevice) != cudaSuccess) {
    delete s;
    return fail(LXW_ERR_CUDA, "lxw_solver_create: upload failed");
  }
  s->dm.hmin_p = d_hp;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
  lxw_status ts = build_tiles(s);
  if (ts != LXW_OK) { delete s; return ts; }
  (void)hmin;
  *out = s;
  return LXW_OK;
}

lxw_status lxw_solver_create(const lxw_mesh* mesh, int degree, const lxw_options* opt, void* stream,
                             lxw_solver** out) {
  if (!mesh) return fail(LXW_ERR_ARG, "lxw_solver_create: null mesh");
  return create_impl(mesh, std::vector<int>{0, mesh->N}, degree, opt, stream, out);
}

lxw_status lxw_batch_create(int nmesh, const lxw_mesh* const* meshes, int degree, const lxw_options* opt,
                            void* stream, lxw_solver** out) {
  if (nmesh < 1 || !meshes || !out) return fail(LXW_ERR_ARG, "lxw_batch_create: bad argument");
  lxw_options o;
  if (opt) o = *opt; else lxw_options_default(&o);
  if (o.precision != LXW_PREC_MIXED && nmesh > 1)
    return fail(LXW_ERR_ARG, "lxw_batch_create: batches of several problems need the mixed precision form");
  lxw_mesh u;
  u.kind = meshes[0] ? meshes[0]->kind : 0; u.E = meshes[0] ? meshes[0]->E : 0; u.N = 0;
  std::vector<int> pstart(1, 0);
  for (int p = 0; p < nmesh; ++p) {
    const lxw_mesh* m = meshes[p];
    if (!m || m->kind != u.kind) return fail(LXW_ERR_ARG, "lxw_batch_create: meshes must exist and share the element kind");
    const int off = u.N;
    u.vx.insert(u.vx.end(), m->vx.begin(), m->vx.end());
    for (size_t k = 0; k < m->nbr.size(); ++k) {
      u.nbr.push_back(m->nbr[k] >= 0 ? m->nbr[k] + off : m->nbr[k]);
      u.nbk.push_back(m->nbk[k]);
    }
    u.N += m->N;
    pstart.push_back(u.N);
  }
  return create_impl(&u, pstart, degree, &o, stream, out);
}

// work list of the mixed kernels: tiles of at most block_threads elements,
// never spanning two problems
static lxw_status build_tiles(lxw_solver* s) {
  const int T = s->opt.block_threads;
  std::vector<int4> tl;
  for (size_t p = 0; p + 1 < s->pstart.size(); ++p)
    for (int a = s->pstart[p]; a < s->pstart[p + 1]; a += T)
      tl.push_back(make_int4(a, std::min(T, s->pstart[p + 1] - a), (int)p, 0));
  if ((int)tl.size() > s->tiles_cap) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(int4) * tl.size()) != cudaSuccess) return fail(LXW_ERR_NOMEM, "tile list allocation failed");
    s->allocs.push_back(p);
    s->d_tiles = (int4*)p;
    s->tiles_cap = (int)tl.size();
  }
  if (cudaMemcpy(s->d_tiles, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(LXW_ERR_CUDA, "tile list upload failed");
  s->dm.tiles = s->d_tiles;
  s->dm.ntiles = (int)tl.size();
  return LXW_OK;
}

void lxw_solver_destroy(lxw_solver* s) { delete s; }

lxw_status lxw_solver_set_stream(lxw_solver* s, void* stream) {
  if (!s) return fail(LXW_ERR_ARG, "lxw_solver_set_stream: null solver");
  s->stream = (cudaStream_t)stream;
  return LXW_OK;
}

lxw_status lxw_solver_info(const lxw_solver* s, int* N, int* E, int* ML, int* npts, int* nproj) {
  if (!s) return fail(LXW_ERR_ARG, "lxw_solver_info: null solver");
  if (N) *N = s->N;
  if (E) *E = s->E;
  if (ML) *ML = s->ML;
  if (npts) *npts = s->tab.NPT;
  if (nproj) *nproj = s->ptab.NPJ;
  return LXW_OK;
}

lxw_status lxw_projection_points(const lxw_solver* s, double* xy) {
  if (!s || !xy) return fail(LXW_ERR_ARG, "lxw_projection_points: null argument");
  std::memcpy(xy, s->xproj.data(), sizeof(double) * s->xproj.size());
  return LXW_OK;
}

lxw_status lxw_basis_eval(int kind, int degree, int n, const double* ref_xy, double* phi) {
  if ((kind != LXW_KIND_QUAD && kind != LXW_KIND_TRI) || (degree != 2 && degree != 3) || n < 0 ||
      (n > 0 && (!ref_xy || !phi)))
    return fail(LXW_ERR_ARG, "lxw_basis_eval: bad argument");
  const int ML = (degree + 1) * (degree + 2) / 2;
  const TriBasis tb = kind == LXW_KIND_TRI ? triangle_basis(ML) : TriBasis{};
  for (int k = 0; k < n; ++k)
    basis_at(kind, ML, tb, ref_xy[2 * k], ref_xy[2 * k + 1], phi + (size_t)k * ML, nullptr, nullptr);
  return LXW_OK;
}

lxw_status lxw_project(lxw_solver* s, const double* prim, double* Q) {
  if (!s || !prim || !Q) return fail(LXW_ERR_ARG, "lxw_project: null argument");
  if (launch_project(s->ptab, s->N, s->opt.gamma, prim, Q, s->stream)) return fail(LXW_ERR_CUDA, "lxw_project: launch failed");
  return LXW_OK;
}

static StepArgs make_args(const lxw_solver* s, double dt, double cfl, int want_diag, double* tc, double* te) {
  StepArgs a{};
  a.dt_in = dt; a.cfl = cfl; a.gamma = s->opt.gamma; a.eps0 = s->opt.eps0; a.alpha0 = s->opt.alpha0;
  a.shock_limiter = s->opt.shock_limiter; a.want_diag = want_diag; a.theta_cell = tc; a.theta_edge = te;
  a.moment_exact = s->opt.moment_exact;
  a.llf_global = s->opt.llf_global;
  a.ck_order = s->opt.ck_order;
  a.gate_scan = s->opt.gate_scan;
  a.gamma_f = (float)a.gamma; a.eps0_f = (float)a.eps0; a.alpha0_f = (float)a.alpha0;
  a.grid = s->opt.ctas_per_sm > 0 ? s->opt.ctas_per_sm * s->sms : 0;   // persistent CTAs, or one per tile
  a.sms = s->sms;
  a.hi_occupancy = s->opt.high_occupancy;
  a.gate_per_sm = s->gate_per_sm[s->opt.high_occupancy ? 1 : 0];
  a.gate_w = s->mlp_w; a.mlp_tau = s->mlp_tau; a.feat_out = nullptr; a.gate_out = nullptr;
  a.gate_wait_test = s->gate_wait_test;
  {  // inflow state and its fluxes (the time-averaged flux of a steady state)
    const double* q = s->qin;
    const double u = q[0] > 0.0 ? q[1] / q[0] : 0.0, v = q[0] > 0.0 ? q[2] / q[0] : 0.0;
    const double p = (a.gamma - 1.0) * (q[3] - 0.5 * (q[1] * u + q[2] * v));
    const double F[4] = {q[1], q[1] * u + p, q[1] * v, (q[3] + p) * u};
    const double G[4] = {q[2], q[2] * u, q[2] * v + p, (q[3] + p) * v};
    for (int k = 0; k < 4; ++k) {
      a.qin[k] = q[k]; a.fin[k] = F[k]; a.gin[k] = G[k];
      a.qin32[k] = (float)q[k]; a.fin32[k] = (float)F[k]; a.gin32[k] = (float)G[k];
    }
  }
  return a;
}

static int do_step(lxw_solver* s, double* Q, const StepArgs& a, cudaStream_t st, void** ev = nullptr,
                   int upto = 99) {
  if (s->mixed) return launch_step_mx(s->kind, s->deg, s->dm, s->dwm, Q, a, st, s->opt.block_threads, ev, upto);
  return launch_step(s->kind, s->deg, s->dm, s->dw, Q, a, st, s->opt.block_threads, ev, upto);
}

static lxw_status read_diag(lxw_solver* s, double dt, double cfl, lxw_diag* d) {
  double* h = s->host_diag;
  LXW_CUDA(cudaMemcpyAsync(h, s->dw.diag, sizeof(DiagBlock), cudaMemcpyDeviceToHost, s->stream));
  LXW_CUDA(cudaMemcpyAsync(h + 32, s->dw.smax, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->stream));
  LXW_CUDA(cudaMemcpyAsync(h + 33, s->dw.status, sizeof(unsigned int), cudaMemcpyDeviceToHost, s->stream));
  LXW_CUDA(cudaStreamSynchronize(s->stream));
  double v[9];
  decode_diag(h, v);
  std::memset(d, 0, sizeof(*d));
  double sp;
  std::memcpy(&sp, h + 32, sizeof(double));
  unsigned int st;
  std::memcpy(&st, h + 33, sizeof(unsigned int));
  d->s = sp;
  d->dt = dt > 0.0 ? dt : cfl * s->dm.hmin / sp;
  if (s->mixed) {
    // largest wave speed and smallest time step over the problems
    std::vector<ScalMx> sc(s->dm.nprob);
    LXW_CUDA(cudaMemcpy(sc.data(), s->dwm.scal, sizeof(ScalMx) * sc.size(), cudaMemcpyDeviceToHost));
    d->s = 0.0; d->dt = 1e300;
    for (const ScalMx& c : sc) { d->s = std::max(d->s, c.s); d->dt = std::min(d->dt, c.dt); }
  }
  d->mass = v[0]; d->momx = v[1]; d->momy = v[2]; d->energy = v[3];
  d->min_rho = v[4]; d->min_p = v[5];
  d->n_mom = v[6]; d->n_edge = v[7]; d->n_sc = v[8];
  d->status = (int)st;
  if (st) LXW_CUDA(cudaMemsetAsync(s->dw.status, 0, sizeof(unsigned int), s->stream));   // reported: clear
  const DiagBlock* blk = reinterpret_cast<const DiagBlock*>(h);
  d->n_fp64_moment = (double)blk->fb_mom;
  d->n_fp64_edge = (double)blk->fb_edge;
  d->n_mlp_skip = (double)blk->mlp_skip;
  if (st & LXW_ST_NONPOSITIVE) return fail(LXW_ERR_NONPOSITIVE, "lxw_step: non-positive cell average at step start");
  if (st & LXW_ST_CFL) return fail(LXW_ERR_CFL, "lxw_step: Gamma^rho < 0 (dt above the low-order CFL bound)");
  if (st & LXW_ST_NAN) return fail(LXW_ERR_NAN, "lxw_step: non-finite state");
  if (st & LXW_ST_TIMEOUT) return fail(LXW_ERR_TIMEOUT, "lxw_step: a device wait of the learned gate gave up");
  return LXW_OK;
}

lxw_status lxw_step(lxw_solver* s, double* Q, double dt, double cfl, lxw_diag* diag, double* theta_cell,
                    double* theta_edge) {
  if (!s || !Q) return fail(LXW_ERR_ARG, "lxw_step: null argument");
  if (!(dt > 0.0) && !(cfl > 0.0)) return fail(LXW_ERR_ARG, "lxw_step: need dt > 0 or cfl > 0");
  StepArgs a = make_args(s, dt, cfl, diag != nullptr, theta_cell, theta_edge);
  if (do_step(s, Q, a, s->stream))
    return fail(LXW_ERR_CUDA, std::string("lxw_step: launch failed: ") + cudaGetErrorString(cudaGetLastError()));
  if (diag) return read_diag(s, dt, cfl, diag);
  return LXW_OK;
}

lxw_status lxw_run(lxw_solver* s, double* Q, int nsteps, double cfl, lxw_diag* diag) {
  if (!s || !Q || nsteps < 0) return fail(LXW_ERR_ARG, "lxw_run: bad argument");
  if (!(cfl > 0.0)) return fail(LXW_ERR_ARG, "lxw_run: cfl must be positive");
  if (nsteps == 0) return LXW_OK;
  int body = diag ? nsteps - 1 : nsteps;
  if (body > 0) {
    if (!s->graph || s->graph_Q != Q || s->graph_cfl != cfl) {
      if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
      StepArgs a = make_args(s, 0.0, cfl, 0, nullptr, nullptr);
      cudaGraph_t g = nullptr;
      LXW_CUDA(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
      int rc = do_step(s, Q, a, s->cap_stream);
      cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &g);
      if (rc || ce != cudaSuccess) { if (g) cudaGraphDestroy(g); return fail(LXW_ERR_CUDA, "lxw_run: graph capture failed"); }
      cudaError_t ie = cudaGraphInstantiate(&s->graph, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) { s->graph = nullptr; return fail(LXW_ERR_CUDA, "lxw_run: graph instantiation failed"); }
      s->graph_Q = Q; s->graph_cfl = cfl;
    }
    for (int k = 0; k < body; ++k) LXW_CUDA(cudaGraphLaunch(s->graph, s->stream));
  }
  if (diag) return lxw_step(s, Q, 0.0, cfl, diag, nullptr, nullptr);
  return LXW_OK;
}

lxw_status lxw_run_to(lxw_solver* s, double* Q, double t_span, double cfl, int max_steps, lxw_diag* diag,
                      int* steps_out, double* t_out) {
  if (!s || !Q || !(t_span > 0.0) || !std::isfinite(t_span) || !(cfl > 0.0) || max_steps < 1)
    return fail(LXW_ERR_ARG, "lxw_run_to: need Q, t_span > 0, cfl > 0 and max_steps >= 1");
  const int nprob = s->dm.nprob > 0 ? s->dm.nprob : 1;
  if (s->mixed && nprob > 1 && s->mlp_w)
    return fail(LXW_ERR_ARG, "lxw_run_to: a batch with the learned gate cannot run to a time");
  StepArgs a = make_args(s, 0.0, cfl, 0, nullptr, nullptr);
  a.timed = 1; a.t_end = t_span; a.tclock = s->tclock;
  LXW_CUDA(cudaMemsetAsync(s->tclock, 0, sizeof(double) * 4 * nprob, s->stream));
  if (!s->tgraph || s->tgraph_Q != Q || s->tgraph_cfl != cfl || s->tgraph_tend != t_span) {
    if (s->tgraph) { cudaGraphExecDestroy(s->tgraph); s->tgraph = nullptr; }
    cudaGraph_t g = nullptr;
    LXW_CUDA(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = do_step(s, Q, a, s->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &g);
    if (rc || ce != cudaSuccess) { if (g) cudaGraphDestroy(g); return fail(LXW_ERR_CUDA, "lxw_run_to: graph capture failed"); }
    cudaError_t ie = cudaGraphInstantiate(&s->tgraph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) { s->tgraph = nullptr; return fail(LXW_ERR_CUDA, "lxw_run_to: graph instantiation failed"); }
    s->tgraph_Q = Q; s->tgraph_cfl = cfl; s->tgraph_tend = t_span;
  }
  // replay in chunks, one synchronisation per chunk: the first chunk is one
  // step (it shows the time step), then enough for the slowest problem at
  // its mean step so far (+5 %); replays after a problem's clock reached
  // t_span cost a few empty launches
  int launched = 0, chunk = 1;
  double tmin = 0.0, smax_steps = 0.0;
  while (launched < max_steps) {
    const int n = std::min(chunk, max_steps - launched);
    for (int k = 0; k < n; ++k) LXW_CUDA(cudaGraphLaunch(s->tgraph, s->stream));
    launched += n;
    LXW_CUDA(cudaMemcpyAsync(s->host_clock, s->tclock, sizeof(double) * 4 * nprob, cudaMemcpyDeviceToHost, s->stream));
    LXW_CUDA(cudaStreamSynchronize(s->stream));
    tmin = 1e300; smax_steps = 0.0;
    double need = 0.0;
    for (int p = 0; p < nprob; ++p) {
      const double t = s->host_clock[4 * p], k = s->host_clock[4 * p + 1];
      tmin = std::min(tmin, t);
      smax_steps = std::max(smax_steps, k);
      if (t < t_span) need = std::max(need, k > 0.0 && t > 0.0 ? (t_span - t) / (t / k) : 1.0);
    }
    if (tmin >= t_span) break;
    chunk = (int)std::min(1e9, std::ceil(1.05 * need)) + 1;
  }
  if (steps_out) *steps_out = (int)smax_steps;
  if (t_out) *t_out = tmin;
  if (diag) {
    // one more timed step with diagnostics: every problem has finished, so
    // its kernels skip; the totals and minima are the final state's, s and
    // dt those of the last step taken, the status the bits seen in the run
    a.want_diag = 1;
    if (do_step(s, Q, a, s->stream)) return fail(LXW_ERR_CUDA, "lxw_run_to: diagnostic launch failed");
    lxw_status st = read_diag(s, 0.0, cfl, diag);
    diag->s = 0.0; diag->dt = 1e300;
    for (int p = 0; p < nprob; ++p) {
      diag->dt = std::min(diag->dt, s->host_clock[4 * p + 2]);
      diag->s = std::max(diag->s, s->host_clock[4 * p + 3]);
    }
    diag->n_mom = diag->n_edge = diag->n_sc = 0.0;
    return st;
  }
  return LXW_OK;
}

lxw_status lxw_run_host(lxw_solver* s, double* Qh, int nsteps, double cfl, lxw_diag* diag) {
  if (!s || !Qh) return fail(LXW_ERR_ARG, "lxw_run_host: null argument");
  const size_t bytes = sizeof(double) * (size_t)s->N * 4 * s->ML;
  // pinned host memory is mapped into the device's address space: the mixed
  // form's pack / unpack kernels then read and write it directly (one pass
  // over the host link each way, no staging copy); pageable memory is copied
  cudaPointerAttributes pa{};
  double* mapped = nullptr;
  if (s->mixed && cudaPointerGetAttributes(&pa, Qh) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
      pa.devicePointer != nullptr)
    mapped = static_cast<double*>(pa.devicePointer);
  cudaGetLastError();   // a pageable pointer may leave an error code behind
  double* state = s->Qdev;
  if (s->mixed) {
    if (!mapped) LXW_CUDA(cudaMemcpyAsync(s->Qdev, Qh, bytes, cudaMemcpyHostToDevice, s->stream));
    if (launch_pack(s->ML, s->N, mapped ? mapped : s->Qdev, s->Sdev, s->stream))
      return fail(LXW_ERR_CUDA, "lxw_run_host: pack failed");
    state = s->Sdev;
  } else {
    LXW_CUDA(cudaMemcpyAsync(s->Qdev, Qh, bytes, cudaMemcpyHostToDevice, s->stream));
  }
  lxw_status st = lxw_run(s, state, nsteps, cfl, diag);
  if (st != LXW_OK && st != LXW_ERR_NONPOSITIVE && st != LXW_ERR_CFL && st != LXW_ERR_NAN && st != LXW_ERR_TIMEOUT)
    return st;
  if (s->mixed) {
    if (launch_unpack(s->ML, s->N, s->Sdev, mapped ? mapped : s->Qdev, s->stream))
      return fail(LXW_ERR_CUDA, "lxw_run_host: unpack failed");
    if (!mapped) LXW_CUDA(cudaMemcpyAsync(Qh, s->Qdev, bytes, cudaMemcpyDeviceToHost, s->stream));
  } else {
    LXW_CUDA(cudaMemcpyAsync(Qh, s->Qdev, bytes, cudaMemcpyDeviceToHost, s->stream));
  }
  LXW_CUDA(cudaStreamSynchronize(s->stream));
  return st;
}

lxw_status lxw_run_host_state(lxw_solver* s, void* state_host, int nsteps, double cfl, lxw_diag* diag) {
  if (!s || !state_host) return fail(LXW_ERR_ARG, "lxw_run_host_state: null argument");
  const size_t bytes = lxw_state_bytes(s);
  double* state = s->mixed ? s->Sdev : s->Qdev;
  LXW_CUDA(cudaMemcpyAsync(state, state_host, bytes, cudaMemcpyHostToDevice, s->stream));
  lxw_status st = lxw_run(s, state, nsteps, cfl, diag);
  if (st != LXW_OK && st != LXW_ERR_NONPOSITIVE && st != LXW_ERR_CFL && st != LXW_ERR_NAN && st != LXW_ERR_TIMEOUT)
    return st;
  LXW_CUDA(cudaMemcpyAsync(state_host, state, bytes, cudaMemcpyDeviceToHost, s->stream));
  LXW_CUDA(cudaStreamSynchronize(s->stream));
  return st;
}

size_t lxw_state_bytes(const lxw_solver* s) {
  if (!s) return 0;
  if (s->mixed) return sizeof(double) * 4 * (size_t)s->N + sizeof(float) * 4 * (size_t)s->ML * s->N;
  return sizeof(double) * 4 * (size_t)s->ML * s->N;
}

lxw_status lxw_state_pack(lxw_solver* s, const double* Q64, void* state) {
  if (!s || !Q64 || !state) return fail(LXW_ERR_ARG, "lxw_state_pack: null argument");
  if (!s->mixed) {
    LXW_CUDA(cudaMemcpyAsync(state, Q64, lxw_state_bytes(s), cudaMemcpyDeviceToDevice, s->stream));
    return LXW_OK;
  }
  if (launch_pack(s->ML, s->N, Q64, (double*)state, s->stream)) return fail(LXW_ERR_CUDA, "lxw_state_pack: launch failed");
  return LXW_OK;
}

lxw_status lxw_state_unpack(lxw_solver* s, const void* state, double* Q64) {
  if (!s || !Q64 || !state) return fail(LXW_ERR_ARG, "lxw_state_unpack: null argument");
  if (!s->mixed) {
    LXW_CUDA(cudaMemcpyAsync(Q64, state, lxw_state_bytes(s), cudaMemcpyDeviceToDevice, s->stream));
    return LXW_OK;
  }
  if (launch_unpack(s->ML, s->N, (const double*)state, Q64, s->stream))
    return fail(LXW_ERR_CUDA, "lxw_state_unpack: launch failed");
  return LXW_OK;
}

lxw_status lxw_moment_limit(lxw_solver* s, double* Q, double* theta, double* s_dev) {
  if (!s || !Q) return fail(LXW_ERR_ARG, "lxw_moment_limit: null argument");
  StepArgs a = make_args(s, 0.0, 0.0, 0, nullptr, nullptr);
  int rc = s->mixed ? launch_moment_limit_mx(s->kind, s->deg, s->dm, s->dwm, Q, a, theta, s->stream, s->opt.block_threads)
                    : launch_moment_limit(s->kind, s->deg, s->dm, s->dw, Q, a, theta, s->stream, s->opt.block_threads);
  if (rc) return fail(LXW_ERR_CUDA, "lxw_moment_limit: launch failed");
  if (s_dev) {
    // the mixed moment kernel leaves each problem's s in its scalars (and clears the maximum)
    if (s->mixed)
      LXW_CUDA(cudaMemcpyAsync(s_dev, &s->dwm.scal[0].s, sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    else if (launch_copy_speed(s->dw, s_dev, s->stream))
      return fail(LXW_ERR_CUDA, "lxw_moment_limit: launch failed");
  }
  return LXW_OK;
}

lxw_status lxw_shock_limit(lxw_solver* s, double* Q, double* theta) {
  if (!s || !Q) return fail(LXW_ERR_ARG, "lxw_shock_limit: null argument");
  if (s->mixed) return fail(LXW_ERR_ARG, "lxw_shock_limit: the mixed form runs the shock limiter inside lxw_step only");
  StepArgs a = make_args(s, 0.0, 0.0, 0, nullptr, nullptr);
  if (launch_shock_limit(s->kind, s->deg, s->dm, Q, a, theta, s->stream, s->opt.block_threads))
    return fail(LXW_ERR_CUDA, "lxw_shock_limit: launch failed");
  return LXW_OK;
}

// the mixed form always launches its shock kernel (it also commits the new averages)
// timed intervals of lxw_profile_step: mixed form moment (+ scalars), ck, edge,
// update, shock (+ gate); FP64 form one per kernel
static int phases_of(const lxw_solver* s) { return s->mixed ? 5 : step_launch_count(0, s->opt.shock_limiter); }
int lxw_profile_phases(const lxw_solver* s) { return s ? phases_of(s) : 0; }
int lxw_step_launches(const lxw_solver* s) {
  if (!s) return 0;
  if (!s->mixed) return step_launch_count(0, s->opt.shock_limiter);
  // moment, ck, edge, update, shock; with the learned gate in its list form
  // the shock phase is two launches (screen + list, gate on the list)
  return s->mlp_w && s->opt.shock_limiter && !s->opt.gate_scan ? 6 : 5;
}

lxw_status lxw_batch_scalars(lxw_solver* s, int* nprob, double* s_host, double* dt_host) {
  if (!s) return fail(LXW_ERR_ARG, "lxw_batch_scalars: null solver");
  if (nprob) *nprob = s->dm.nprob;
  if (!s_host && !dt_host) return LXW_OK;
  if (!s->mixed) return fail(LXW_ERR_ARG, "lxw_batch_scalars: needs the mixed form");
  LXW_CUDA(cudaStreamSynchronize(s->stream));
  std::vector<ScalMx> sc(s->dm.nprob);
  LXW_CUDA(cudaMemcpy(sc.data(), s->dwm.scal, sizeof(ScalMx) * sc.size(), cudaMemcpyDeviceToHost));
  for (size_t p = 0; p < sc.size(); ++p) {
    if (s_host) s_host[p] = sc[p].s;
    if (dt_host) dt_host[p] = sc[p].dt;
  }
  return LXW_OK;
}

lxw_status lxw_solver_set_mlp(lxw_solver* s, lxw_mlp* mlp, float tau) {
  if (!s) return fail(LXW_ERR_ARG, "lxw_solver_set_mlp: null solver");
  if (!s->mixed) return fail(LXW_ERR_ARG, "lxw_solver_set_mlp: the learned gate needs the mixed form");
  if (!(tau >= 0.0f && tau < 1.0f)) return fail(LXW_ERR_ARG, "lxw_solver_set_mlp: tau must be in [0, 1)");
  if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
  if (s->pgraph) { cudaGraphExecDestroy(s->pgraph); s->pgraph = nullptr; }
  if (!mlp) { s->mlp_w = nullptr; return LXW_OK; }
  if (!s->gate_buf) {
    void* p = nullptr;
    LXW_CUDA(cudaMalloc(&p, sizeof(GateWeights)));
    s->allocs.push_back(p);
    s->gate_buf = (GateWeights*)p;
  }
  if (mlp_gate_weights(mlp, s->gate_buf)) return fail(LXW_ERR_CUDA, "lxw_solver_set_mlp: weight layout failed");
  for (int hi = 0; hi < 2; ++hi) {
    const int occ = gate_occupancy(s->kind, s->deg, hi);
    if (occ < 1) return fail(LXW_ERR_CUDA, "lxw_solver_set_mlp: the gate kernel does not fit on this device");
    s->gate_per_sm[hi] = occ;
  }
  s->mlp_w = s->gate_buf;
  s->mlp_tau = tau;
  return LXW_OK;
}

lxw_status lxw_step_dump(lxw_solver* s, void* state, double cfl, float* feat, double* theta_sc) {
  if (!s || !state || !feat || !(cfl > 0.0)) return fail(LXW_ERR_ARG, "lxw_step_dump: bad argument");
  if (!s->mixed) return fail(LXW_ERR_ARG, "lxw_step_dump: needs the mixed form");
  if (!s->opt.shock_limiter) return fail(LXW_ERR_ARG, "lxw_step_dump: the shock limiter is off");
  // theta_cell is [2][N] (moment, shock); a scratch pair keeps the shock row
  void* scratch = nullptr;
  if (theta_sc) LXW_CUDA(cudaMalloc(&scratch, sizeof(double) * 2 * (size_t)s->N));
  StepArgs a = make_args(s, 0.0, cfl, 0, (double*)scratch, nullptr);
  a.gate_w = nullptr;                      // the plain limiter labels the data
  a.feat_out = feat;
  int rc = do_step(s, (double*)state, a, s->stream);
  if (!rc && theta_sc)
    cudaMemcpyAsync(theta_sc, (double*)scratch + s->N, sizeof(double) * s->N, cudaMemcpyDeviceToDevice, s->stream);
  cudaError_t se = cudaStreamSynchronize(s->stream);
  if (scratch) cudaFree(scratch);
  if (rc || se != cudaSuccess) return fail(LXW_ERR_CUDA, "lxw_step_dump: launch failed");
  return LXW_OK;
}

lxw_status lxw_step_gate(lxw_solver* s, void* state, double cfl, float* gate, float* feat) {
  if (!s || !state || !gate || !(cfl > 0.0)) return fail(LXW_ERR_ARG, "lxw_step_gate: bad argument");
  if (!s->mixed) return fail(LXW_ERR_ARG, "lxw_step_gate: needs the mixed form");
  if (!s->opt.shock_limiter) return fail(LXW_ERR_ARG, "lxw_step_gate: the shock limiter is off");
  if (!s->mlp_w) return fail(LXW_ERR_ARG, "lxw_step_gate: no network attached (lxw_solver_set_mlp)");
  // all-ones bytes are a NaN: cells whose averages fail the positivity check get no theta_hat
  LXW_CUDA(cudaMemsetAsync(gate, 0xff, sizeof(float) * (size_t)s->N, s->stream));
  StepArgs a = make_args(s, 0.0, cfl, 0, nullptr, nullptr);
  a.gate_out = gate;
  a.feat_out = feat;
  int rc = do_step(s, (double*)state, a, s->stream);
  cudaError_t se = cudaStreamSynchronize(s->stream);
  if (rc || se != cudaSuccess) return fail(LXW_ERR_CUDA, "lxw_step_gate: launch failed");
  return LXW_OK;
}

static void drop_graphs(lxw_solver* s) {
  if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
  if (s->tgraph) { cudaGraphExecDestroy(s->tgraph); s->tgraph = nullptr; }
  if (s->pgraph) { cudaGraphExecDestroy(s->pgraph); s->pgraph = nullptr; }
}

lxw_status lxw_solver_set_inflow(lxw_solver* s, const double prim[4]) {
  if (!s || !prim) return fail(LXW_ERR_ARG, "lxw_solver_set_inflow: null argument");
  if (!(prim[0] > 0.0) || !(prim[3] > 0.0) || !std::isfinite(prim[1]) || !std::isfinite(prim[2]))
    return fail(LXW_ERR_ARG, "lxw_solver_set_inflow: needs rho > 0, p > 0 and finite velocity");
  s->qin[0] = prim[0];
  s->qin[1] = prim[0] * prim[1];
  s->qin[2] = prim[0] * prim[2];
  s->qin[3] = prim[3] / (s->opt.gamma - 1.0) + 0.5 * prim[0] * (prim[1] * prim[1] + prim[2] * prim[2]);
  drop_graphs(s);
  return LXW_OK;
}

lxw_status lxw_solver_set_gate_wait_test(lxw_solver* s, long long cycles) {
  if (!s || cycles < 0) return fail(LXW_ERR_ARG, "lxw_solver_set_gate_wait_test: null solver or negative cycles");
  s->gate_wait_test = cycles;
  drop_graphs(s);
  return LXW_OK;
}

lxw_status lxw_autotune(lxw_solver* s, void* state, double cfl, int reps, int* bt, int* cps, float* best_ms,
                        int* hiocc) {
  if (!s || !state || !(cfl > 0.0) || reps < 1) return fail(LXW_ERR_ARG, "lxw_autotune: bad argument");
  const size_t bytes = lxw_state_bytes(s);
  void* save = nullptr;
  LXW_CUDA(cudaStreamSynchronize(s->stream));
  LXW_CUDA(cudaMalloc(&save, bytes));
  LXW_CUDA(cudaMemcpy(save, state, bytes, cudaMemcpyDeviceToDevice));
  const int blocks[3] = {32, 64, 128};
  const int ctas[7] = {0, 1, 2, 3, 4, 6, 8};
  const lxw_options keep = s->opt;
  float best = 1e30f;
  int bb = keep.block_threads, bc = keep.ctas_per_sm, bh = keep.high_occupancy;
  lxw_status st = LXW_OK;
  float ms[8];
  for (int hi = 0; hi < (s->mixed ? 2 : 1) && st == LXW_OK; ++hi)
  for (int b : blocks) {
    for (int c : ctas) {
      if (!s->mixed && c != 0) continue;
      s->opt.block_threads = b; s->opt.ctas_per_sm = c; s->opt.high_occupancy = hi;
      drop_graphs(s);
      if ((st = build_tiles(s)) != LXW_OK) break;
      cudaMemcpy(state, save, bytes, cudaMemcpyDeviceToDevice);
      if ((st = lxw_profile_step(s, (double*)state, cfl, ms)) != LXW_OK) break;   // warm-up + capture
      float tot = 0.0f;
      for (int r = 0; r < reps; ++r) {
        if ((st = lxw_profile_step(s, (double*)state, cfl, ms)) != LXW_OK) break;
        for (int k = 0; k < phases_of(s); ++k) tot += ms[k];
      }
      if (st != LXW_OK) break;
      if (tot / reps < best) { best = tot / reps; bb = b; bc = c; bh = hi; }
    }
    if (st != LXW_OK) break;
  }
  s->opt.block_threads = bb; s->opt.ctas_per_sm = bc; s->opt.high_occupancy = bh;
  if (st == LXW_OK && s->mixed && s->mlp_w && s->opt.shock_limiter) {
    // the gated limiter's two forms, on the chosen work list
    if ((st = build_tiles(s)) == LXW_OK) {
      float bt[2] = {1e30f, 1e30f};
      for (int g = 0; g < 2 && st == LXW_OK; ++g) {
        s->opt.gate_scan = g;
        drop_graphs(s);
        cudaMemcpy(state, save, bytes, cudaMemcpyDeviceToDevice);
        if ((st = lxw_profile_step(s, (double*)state, cfl, ms)) != LXW_OK) break;
        float tot = 0.0f;
        for (int r = 0; r < reps && st == LXW_OK; ++r) {
          if ((st = lxw_profile_step(s, (double*)state, cfl, ms)) != LXW_OK) break;
          for (int k = 0; k < phases_of(s); ++k) tot += ms[k];
        }
        bt[g] = tot / reps;
      }
      s->opt.gate_scan = bt[1] < bt[0] ? 1 : 0;
      best = std::min(bt[0], bt[1]);
    }
  }
  drop_graphs(s);
  lxw_status tst = build_tiles(s);
  cudaMemcpy(state, save, bytes, cudaMemcpyDeviceToDevice);
  cudaFree(save);
  if (st != LXW_OK) return st;
  if (tst != LXW_OK) return tst;
  if (bt) *bt = bb;
  if (cps) *cps = bc;
  if (best_ms) *best_ms = best;
  if (hiocc) *hiocc = bh;
  return LXW_OK;
}

lxw_status lxw_solver_get_options(const lxw_solver* s, lxw_options* out) {
  if (!s || !out) return fail(LXW_ERR_ARG, "lxw_solver_get_options: null argument");
  *out = s->opt;
  return LXW_OK;
}

lxw_status lxw_step_phases(lxw_solver* s, double* Q, double dt, double cfl, int nphases) {
  if (!s || !Q || nphases < 1) return fail(LXW_ERR_ARG, "lxw_step_phases: bad argument");
  if (!(dt > 0.0) && !(cfl > 0.0)) return fail(LXW_ERR_ARG, "lxw_step_phases: need dt > 0 or cfl > 0");
  StepArgs a = make_args(s, dt, cfl, 0, nullptr, nullptr);
  s->last_dt_in = dt; s->last_cfl = cfl;
  if (do_step(s, Q, a, s->stream, nullptr, nphases))
    return fail(LXW_ERR_CUDA, "lxw_step_phases: launch failed");
  return LXW_OK;
}

lxw_status lxw_workspace_copy(lxw_solver* s, int which, double* out, size_t count) {
  if (!s || !out) return fail(LXW_ERR_ARG, "lxw_workspace_copy: null argument");
  const size_t N = s->N, E = s->E, MQ = s->tab.MQ;
  const double* src = nullptr;
  size_t n = 0;
  if (s->mixed && (which == 0 || which == 1)) {
    // FP32 buffers: traces [E][MQ][8][N]; f^LxW [E][4][N] returned as [E][8][N] with zero f^LxF
    const size_t nf = which == 0 ? E * MQ * 8 * N : E * 4 * N, nout = which == 0 ? nf : E * 8 * N;
    if (count < nout) return fail(LXW_ERR_ARG, "lxw_workspace_copy: buffer too small");
    std::vector<float> tmp(nf);
    LXW_CUDA(cudaMemcpyAsync(tmp.data(), which == 0 ? (const void*)s->dwm.trace : (const void*)s->dwm.fw,
                             nf * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    LXW_CUDA(cudaStreamSynchronize(s->stream));
    if (which == 0) {
      for (size_t k = 0; k < nf; ++k) out[k] = tmp[k];
    } else {
      for (size_t k = 0; k < E; ++k)
        for (size_t c = 0; c < 8; ++c)
          for (size_t i = 0; i < N; ++i) out[(k * 8 + c) * N + i] = c < 4 ? tmp[(k * 4 + c) * N + i] : 0.0;
    }
    return LXW_OK;
  }
  if (s->mixed && which == 2) {
    if (count < E * N) return fail(LXW_ERR_ARG, "lxw_workspace_copy: buffer too small");
    std::vector<float> tmp(E * N);
    LXW_CUDA(cudaMemcpyAsync(tmp.data(), s->dwm.prop, E * N * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    LXW_CUDA(cudaStreamSynchronize(s->stream));
    for (size_t k = 0; k < E * N; ++k) out[k] = tmp[k];
    return LXW_OK;
  }
  if (which == 0) { src = s->dw.trace; n = E * MQ * 8 * N; }
  else if (which == 1) { src = s->dw.flux; n = E * 8 * N; }
  else if (which == 2) { src = s->dw.prop; n = E * N; }
  else if (which == 3 && s->mixed) {
    if (count < 2) return fail(LXW_ERR_ARG, "lxw_workspace_copy: buffer too small");
    ScalMx sc;
    LXW_CUDA(cudaMemcpyAsync(&sc, s->dwm.scal, sizeof(sc), cudaMemcpyDeviceToHost, s->stream));
    LXW_CUDA(cudaStreamSynchronize(s->stream));
    out[0] = sc.s; out[1] = sc.dt;
    return LXW_OK;
  } else if (which == 3) {
    if (count < 2) return fail(LXW_ERR_ARG, "lxw_workspace_copy: buffer too small");
    unsigned long long b = 0;
    LXW_CUDA(cudaMemcpyAsync(&b, s->dw.smax, sizeof(b), cudaMemcpyDeviceToHost, s->stream));
    LXW_CUDA(cudaStreamSynchronize(s->stream));
    std::memcpy(&out[0], &b, sizeof(double));
    out[1] = s->last_dt_in > 0.0 ? s->last_dt_in : s->last_cfl * s->dm.hmin / out[0];
    return LXW_OK;
  } else {
    return fail(LXW_ERR_ARG, "lxw_workspace_copy: unknown buffer");
  }
  if (count < n) return fail(LXW_ERR_ARG, "lxw_workspace_copy: buffer too small");
  LXW_CUDA(cudaMemcpyAsync(out, src, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  LXW_CUDA(cudaStreamSynchronize(s->stream));
  return LXW_OK;
}

lxw_status lxw_profile_step(lxw_solver* s, double* Q, double cfl, float* ms) {
  if (!s || !Q || !ms || !(cfl > 0.0)) return fail(LXW_ERR_ARG, "lxw_profile_step: bad argument");
  // the step is replayed from a graph with an event node around every kernel,
  // so the intervals are device time without host launch gaps
  if (!s->pgraph || s->pgraph_Q != Q || s->pgraph_cfl != cfl) {
    if (s->pgraph) { cudaGraphExecDestroy(s->pgraph); s->pgraph = nullptr; }
    StepArgs a = make_args(s, 0.0, cfl, 0, nullptr, nullptr);
    cudaGraph_t g = nullptr;
    LXW_CUDA(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = do_step(s, Q, a, s->cap_stream, s->events);
    cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &g);
    if (rc || ce != cudaSuccess) { if (g) cudaGraphDestroy(g); return fail(LXW_ERR_CUDA, "lxw_profile_step: capture failed"); }
    cudaError_t ie = cudaGraphInstantiate(&s->pgraph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) { s->pgraph = nullptr; return fail(LXW_ERR_CUDA, "lxw_profile_step: instantiation failed"); }
    s->pgraph_Q = Q; s->pgraph_cfl = cfl;
  }
  LXW_CUDA(cudaGraphLaunch(s->pgraph, s->stream));
  const int n = phases_of(s);
  LXW_CUDA(cudaEventSynchronize((cudaEvent_t)s->events[n]));
  for (int k = 0; k < n; ++k) LXW_CUDA(cudaEventElapsedTime(&ms[k], (cudaEvent_t)s->events[k], (cudaEvent_t)s->events[k + 1]));
  return LXW_OK;
}

}  // extern "C"
