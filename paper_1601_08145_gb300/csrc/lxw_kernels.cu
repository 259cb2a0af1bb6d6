// lxw_kernels.cu -- sm_103a kernels of one LxW-DG time step (FP64 form).
//
// One thread owns one element.  The quadrature/basis tables travel in the
// kernel-parameter constant bank (all threads of a warp read the same entry
// at the same time), the geometry and every per-element array are stored
// structure-of-arrays [..][N] so that a warp's loads of one field are
// coalesced.  The step is five dependent phases separated by kernel
// boundaries (grid-wide dependencies: a global wave speed, neighbour
// traces, neighbour Lambda proposals, neighbour new averages):
//   k_moment   Sec. 3.1 moment limiter + block max of |u|+c -> atomicMax
//   k_ck       Sec. 2.2-2.3 CK time-averaged flux, volume integral, traces
//   k_edge     Sec. 3.3 Step 3 (LLF, f^LxW, f^LxF, edge integral) and
//              Steps 4-5 (Gamma, Lambda, box corners, mu) per element
//   k_update   Sec. 3.3 Step 6: theta_e = min of both proposals, averages
//   k_shock    Sec. 4.1 shock-capturing limiter on the new state
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "lxw_internal.h"

namespace lxw {
namespace {

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ unsigned long long ordered_bits(double x) {
  // order-preserving map of doubles onto unsigned 64-bit integers
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

// Tables of the four (element kind, degree) variants: 0 quad P2, 1 quad P3,
// 2 triangle P2, 3 triangle P3.  They depend on nothing but the variant, so
// one copy per device serves every solver.
__constant__ Tables c_tabs[4];

struct DevDiag {             // layout of DevWork::diag
  double sum[4];             // sum_i |T_i| qbar_i
  unsigned long long minr, minp;   // ordered bits of min rho, min p
  unsigned long long nmom, nedge, nsc;
};

// A timed run (lxw_run_to) stops each problem when its clock reaches t_end:
// the kernels of a step skip it then, and its last step is shortened to
// land on t_end.  The clock only moves between steps (k_clock).
__device__ __forceinline__ bool step_live(const StepArgs& a) { return !a.timed || __ldcg(a.tclock) < a.t_end; }

__device__ __forceinline__ double step_dt(const DevWork& w, const DevMesh& m, const StepArgs& a) {
  double s = __longlong_as_double((long long)*w.smax);
  double dt = a.dt_in > 0.0 ? a.dt_in : a.cfl * m.hmin / s;
  if (a.timed) {
    const double t = __ldcg(a.tclock);
    if (t + dt >= a.t_end) dt = a.t_end - t;
  }
  return dt;
}

// Euler flux and its directional derivatives (Eqs. 1-2, fluxderivs-a/b).
// Point state with cached primitives.
struct Pt {
  double r, m, n, e;     // conserved
  double ri, u, v, p;    // 1/rho, velocity, pressure
};
__device__ __forceinline__ Pt make_pt(double g1, double r, double m, double n, double e) {
  Pt s;
  s.r = r; s.m = m; s.n = n; s.e = e;
  s.ri = 1.0 / r;
  s.u = m * s.ri; s.v = n * s.ri;
  s.p = g1 * (e - 0.5 * (m * s.u + n * s.v));
  return s;
}
__device__ __forceinline__ void euler_flux(const Pt& s, double F[4], double G[4]) {
  double h = s.e + s.p;
  F[0] = s.m; F[1] = s.m * s.u + s.p; F[2] = s.m * s.v; F[3] = h * s.u;
  G[0] = s.n; G[1] = s.n * s.u; G[2] = s.n * s.v + s.p; G[3] = h * s.v;
}
// first derivative of (F,G) along w; also returns du, dv, dp for reuse
__device__ __forceinline__ void euler_d1(double g1, const Pt& s, const double w[4], double F[4], double G[4],
                                         double& du, double& dv, double& dp) {
  du = (w[1] - s.u * w[0]) * s.ri;
  dv = (w[2] - s.v * w[0]) * s.ri;
  double dK = s.u * w[1] + s.v * w[2] - 0.5 * (s.u * s.u + s.v * s.v) * w[0];
  dp = g1 * (w[3] - dK);
  double h = s.e + s.p, dh = w[3] + dp;
  F[0] = w[1]; F[1] = w[1] * s.u + s.m * du + dp; F[2] = w[1] * s.v + s.m * dv; F[3] = dh * s.u + h * du;
  G[0] = w[2]; G[1] = w[2] * s.u + s.n * du; G[2] = w[2] * s.v + s.n * dv + dp; G[3] = dh * s.v + h * dv;
}
// second derivative of (F,G) along w, given du, dv, dp of the same direction
__device__ __forceinline__ void euler_d2(double g1, const Pt& s, const double w[4], double du, double dv,
                                         double dp, double F[4], double G[4]) {
  double ddu = -2.0 * du * w[0] * s.ri, ddv = -2.0 * dv * w[0] * s.ri;
  double ddp = -g1 * s.r * (du * du + dv * dv);
  double h = s.e + s.p, dh = w[3] + dp;
  F[0] = 0.0; F[1] = 2.0 * w[1] * du + s.m * ddu + ddp; F[2] = 2.0 * w[1] * dv + s.m * ddv;
  F[3] = ddp * s.u + 2.0 * dh * du + h * ddu;
  G[0] = 0.0; G[1] = 2.0 * w[2] * du + s.n * ddu; G[2] = 2.0 * w[2] * dv + s.n * ddv + ddp;
  G[3] = ddp * s.v + 2.0 * dh * dv + h * ddv;
}

// Third derivative of (F, G) along w (a term of the fourth-order time
// average, Sec. 2.2 series continued): the Taylor coefficients in e of u, v,
// p along q + e w by series products (rho u = m gives u_k = (m_k - w_rho
// u_{k-1}) / rho), each flux component's third derivative being 3! times its
// coefficient of e^3.
__device__ __forceinline__ void euler_d3(double g1, const Pt& s, const double w[4], double F[4], double G[4]) {
  const double u1 = (w[1] - s.u * w[0]) * s.ri, v1 = (w[2] - s.v * w[0]) * s.ri;
  const double u2 = -w[0] * u1 * s.ri, v2 = -w[0] * v1 * s.ri;
  const double u3 = -w[0] * u2 * s.ri, v3 = -w[0] * v2 * s.ri;
  // K_3 = (m u_3 + w_m u_2 + n v_3 + w_n v_2) / 2, p_3 = -(g-1) K_3 (E is linear)
  const double p3 = -g1 * 0.5 * (s.m * u3 + w[1] * u2 + s.n * v3 + w[2] * v2);
  const double K2 = 0.5 * (s.m * u2 + w[1] * u1 + s.n * v2 + w[2] * v1);
  const double K1 = 0.5 * (s.m * u1 + w[1] * s.u + s.n * v1 + w[2] * s.v);
  const double p2 = -g1 * K2, p1 = g1 * (w[3] - K1);
  const double H0 = s.e + s.p, H1 = w[3] + p1, H2 = p2, H3 = p3;
  F[0] = 0.0;
  F[1] = 6.0 * (s.m * u3 + w[1] * u2 + p3);
  F[2] = 6.0 * (s.m * v3 + w[1] * v2);
  F[3] = 6.0 * (H0 * u3 + H1 * u2 + H2 * u1 + H3 * s.u);
  G[0] = 0.0;
  G[1] = 6.0 * (s.n * u3 + w[2] * u2);
  G[2] = 6.0 * (s.n * v3 + w[2] * v2 + p3);
  G[3] = 6.0 * (H0 * v3 + H1 * v2 + H2 * v1 + H3 * s.v);
}
// mixed second derivative of (F, G) in the directions a and b, from the
// bilinear chain rule (no cancellation): with u_a = (a_m - u a_rho)/rho, the
// mixed derivative of u is -(u_b a_rho + u_a b_rho)/rho and that of p is
// -(g-1) rho (u_a u_b + v_a v_b); each flux component is a product rule.
__device__ __forceinline__ void euler_d11(double g1, const Pt& s, const double a[4], const double b[4], double F[4],
                                          double G[4]) {
  const double ua = (a[1] - s.u * a[0]) * s.ri, va = (a[2] - s.v * a[0]) * s.ri;
  const double ub = (b[1] - s.u * b[0]) * s.ri, vb = (b[2] - s.v * b[0]) * s.ri;
  const double uab = -(ub * a[0] + ua * b[0]) * s.ri, vab = -(vb * a[0] + va * b[0]) * s.ri;
  const double pa = g1 * (a[3] - (s.u * a[1] + s.v * a[2] - 0.5 * (s.u * s.u + s.v * s.v) * a[0]));
  const double pb = g1 * (b[3] - (s.u * b[1] + s.v * b[2] - 0.5 * (s.u * s.u + s.v * s.v) * b[0]));
  const double pab = -g1 * s.r * (ua * ub + va * vb);
  const double H = s.e + s.p, Ha = a[3] + pa, Hb = b[3] + pb;
  F[0] = 0.0;
  F[1] = a[1] * ub + b[1] * ua + s.m * uab + pab;
  F[2] = a[1] * vb + b[1] * va + s.m * vab;
  F[3] = pab * s.u + Ha * ub + Hb * ua + H * uab;
  G[0] = 0.0;
  G[1] = a[2] * ub + b[2] * ua + s.n * uab;
  G[2] = a[2] * vb + b[2] * va + s.n * vab + pab;
  G[3] = pab * s.v + Ha * vb + Hb * va + H * vab;
}

__device__ __forceinline__ double speed_of(double g, double r, double m, double n, double e) {
  double ri = 1.0 / r;
  double kin2 = m * m + n * n;
  double p = (g - 1.0) * (e - 0.5 * kin2 * ri);
  p = p > 0.0 ? p : 0.0;
  return sqrt(kin2) * ri + sqrt(g * p * ri);
}

// |u| + c of a point state for the dissipation of the LLF point flux, in
// explicitly rounded operations: the two elements of an edge evaluate it on
// the same two traces and must get the same value (their fluxes are exact
// negatives).  A non-positive density gives NaN, which the fmin / fmax that
// combine the speeds discard.
__device__ __forceinline__ double lf_speed(double g, const double q[4]) {
  const double ri = __drcp_rn(q[0]);
  const double kin2 = __fma_rn(q[1], q[1], __dmul_rn(q[2], q[2]));
  double p = __dmul_rn(g - 1.0, __fma_rn(__dmul_rn(-0.5, kin2), ri, q[3]));
  p = p > 0.0 ? p : 0.0;
  return __dadd_rn(__dmul_rn(__dsqrt_rn(kin2), ri), __dsqrt_rn(__dmul_rn(__dmul_rn(g, p), ri)));
}

__device__ __forceinline__ void block_max_to(double v, unsigned long long* dst) {
  // warp shuffle, then one atomic per warp (values are non-negative)
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(dst, (unsigned long long)__double_as_longlong(v));
}

// boundary exterior state for reflective (flip normal momentum) or
// transparent (copy) conditions, Sec. 2.4, or the prescribed inflow state
__device__ __forceinline__ void ghost_state(int bc, double nxh, double nyh, const double qi[4], double qo[4],
                                            const double qin[4]) {
  if (bc == LXW_BC_INFLOW) {
#pragma unroll
    for (int v = 0; v < 4; ++v) qo[v] = qin[v];
    return;
  }
  qo[0] = qi[0]; qo[3] = qi[3];
  if (bc == LXW_BC_REFLECT) {
    double mn = qi[1] * nxh + qi[2] * nyh;
    qo[1] = qi[1] - 2.0 * mn * nxh;
    qo[2] = qi[2] - 2.0 * mn * nyh;
  } else {
    qo[1] = qi[1]; qo[2] = qi[2];
  }
}

// Largest theta in [0, thr] keeping p >= ep at a point whose limited state is
// q(theta) = qbar + theta d (Sec. 3.1: the optimal theta computed exactly).
// h(theta) = (rho p - ep rho)/(g-1) = h0 + h1 theta + h2 theta^2 is positive
// at 0 and negative at thr when it is called, so it has one root in between,
// taken in the cancellation-free form.
__device__ __forceinline__ double exact_root_theta(double rb, double mb, double nb, double eb, const double d[4],
                                                   double kappa, double thr) {
  const double h0 = rb * eb - 0.5 * (mb * mb + nb * nb) - kappa * rb;
  const double h1 = rb * d[3] + d[0] * eb - (mb * d[1] + nb * d[2]) - kappa * d[0];
  const double h2 = d[0] * d[3] - 0.5 * (d[1] * d[1] + d[2] * d[2]);
  const double disc = fmax(h1 * h1 - 4.0 * h0 * h2, 0.0);
  const double den = -h1 + sqrt(disc);
  return den > 0.0 ? fmin(2.0 * h0 / den, thr) : 0.0;
}

// ------------------------------------------------------------ k_reset
__global__ void k_reset(DevWork w, int want_diag, int clear_status) {
  *w.smax = 0ull;
  if (clear_status) *w.status = 0u;
  if (want_diag) {
    DevDiag* d = reinterpret_cast<DevDiag*>(w.diag);
    for (int c = 0; c < 4; ++c) d->sum[c] = 0.0;
    d->minr = d->minp = ~0ull;
    d->nmom = d->nedge = d->nsc = 0ull;
  }
}

// ------------------------------------------------------------ k_clock
// End of a timed step: advance the clock by the step's dt, or set it to
// t_end exactly on the shortened last step.
__global__ void k_clock(const DevMesh m, const DevWork w, const StepArgs a) {
  const double t = a.tclock[0];
  if (!(t < a.t_end)) return;
  const double s = __longlong_as_double((long long)*w.smax);
  const double dt = a.dt_in > 0.0 ? a.dt_in : a.cfl * m.hmin / s;
  const bool last = t + dt >= a.t_end;
  a.tclock[0] = last ? a.t_end : t + dt;
  a.tclock[1] += 1.0;
  a.tclock[2] = last ? a.t_end - t : dt;
  a.tclock[3] = s;
}

// ------------------------------------------------------------ k_moment
// Sec. 3.1 Steps 0-2 (Lemma 1 secant with the density factor), then the
// contribution of this element to the global wave speed s (max of |u|+c
// over the average and the limited point values).
// EXACT: the exact-root variant of the pressure step (a separate instance, so
// that the default one keeps its registers)
template <int KD, int E, int ML, int NQ, int MQ, bool EXACT = false>
__global__ void __launch_bounds__(128) k_moment(const DevMesh m, const DevWork w, double* __restrict__ Q,
                                                const StepArgs a, double* __restrict__ theta_out) {
  constexpr int NPT = NQ + E * MQ;
  const Tables& t = c_tabs[KD];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (!step_live(a)) return;                 // uniform over the grid
  double smax = 0.0;
  if (i < m.N) {
    const double g = a.gamma, g1 = g - 1.0;
    double* Qi = Q + (size_t)i * 4 * ML;
    double c[4][ML];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int l = 0; l < ML; ++l) c[v][l] = Qi[v * ML + l];
    const double rb = c[0][0], mb = c[1][0], nb = c[2][0], eb = c[3][0];
    const double pb = rb > 0.0 ? g1 * (eb - 0.5 * (mb * mb + nb * nb) / rb) : -1.0;
    double th = 1.0;
    if (!(rb > 0.0) || !(pb > 0.0)) {
      atomicOr(w.status, (unsigned)LXW_ST_NONPOSITIVE);
      th = 0.0;
    } else {
      // deviations from the average at every limiter point
      double d[NPT][4];
#pragma unroll
      for (int p = 0; p < NPT; ++p)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          double acc = 0.0;
#pragma unroll
          for (int l = 1; l < ML; ++l) acc = fma(c[v][l], t.phi[p][l], acc);
          d[p][v] = acc;
        }
      // Step 1: density
      const double er = fmin(a.eps0, 0.5 * rb);
      double thr = 1.0;
#pragma unroll
      for (int p = 0; p < NPT; ++p) {
        double rm = rb + d[p][0];
        if (rm < er) thr = fmin(thr, (rb - er) / (rb - rm));
      }
      // Step 2: pressure on the density-limited state, and the speed of that state
      const double ep = fmin(a.eps0, 0.5 * pb);
      th = thr;
#pragma unroll
      for (int p = 0; p < NPT; ++p) {
        double r = rb + thr * d[p][0], mm = mb + thr * d[p][1], nn = nb + thr * d[p][2], ee = eb + thr * d[p][3];
        double ri = 1.0 / r, kin2 = mm * mm + nn * nn;
        double pt = g1 * (ee - 0.5 * kin2 * ri);
        if (pt < ep)
          th = fmin(th, EXACT ? exact_root_theta(rb, mb, nb, eb, d[p], ep / g1, thr) : thr * (pb - ep) / (pb - pt));
        double pp = pt > 0.0 ? pt : 0.0;
        smax = fmax(smax, sqrt(kin2) * ri + sqrt(g * pp * ri));
      }
      th = fmax(th, 0.0);
      if (th < thr) {
        // pressure limiting changed theta: the speeds must be re-evaluated
        smax = 0.0;
#pragma unroll
        for (int p = 0; p < NPT; ++p)
          smax = fmax(smax, speed_of(g, rb + th * d[p][0], mb + th * d[p][1], nb + th * d[p][2], eb + th * d[p][3]));
      }
      smax = fmax(smax, speed_of(g, rb, mb, nb, eb));
    }
    if (th < 1.0) {
#pragma unroll
      for (int v = 0; v < 4; ++v)
#pragma unroll
        for (int l = 1; l < ML; ++l) Qi[v * ML + l] = th * c[v][l];
      if (a.want_diag) atomicAdd(&reinterpret_cast<DevDiag*>(w.diag)->nmom, 1ull);
    }
    if (theta_out) theta_out[i] = th;
  }
  block_max_to(smax, w.smax);
}

// ------------------------------------------------------------ k_ck
// Sec. 2.3 Steps 1-2: Galerkin projection of the (contravariant) flux with
// the interior rule, q_t = -div F^h, F_t = F'(q) q_t, projection, q_tt =
// -div F_t^h, F_tt = F''(q)(q_t,q_t) + F'(q) q_tt, F_T = F + dt/2 F_t +
// dt^2/6 F_tt (Eq. taylor3-flux).  Step 3 interior integral added to the
// higher moments in place: Q^(l) += dt/|T| Int grad phi . F_T.  Edge points
// store q and n_out . F_T for the edge phase.
// ORD4: fourth order in time (one more term of the series): q_ttt = -div
// F_tt^h of the projected contravariant F_tt, F_ttt = F'''(q)(q_t,q_t,q_t) +
// 3 F''(q)(q_t,q_tt) + F'(q) q_ttt, F_T += dt^3/24 F_ttt.
template <int KD, int E, int ML, int NQ, int MQ, bool ORD4 = false>
__global__ void __launch_bounds__(128) k_ck(const DevMesh m, const DevWork w, double* __restrict__ Q,
                                            const StepArgs a) {
  constexpr int NPT = NQ + E * MQ;
  const Tables& t = c_tabs[KD];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N || !step_live(a)) return;
  const int N = m.N;
  const double g1 = a.gamma - 1.0;
  const double dt = step_dt(w, m, a);
  const double c1 = 0.5 * dt, c2 = dt * dt / 6.0;
  double* Qi = Q + (size_t)i * 4 * ML;
  double c[4][ML];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) c[v][l] = Qi[v * ML + l];
  const double jxx = m.jinv[i], jxy = m.jinv[N + i], jyx = m.jinv[2 * N + i], jyy = m.jinv[3 * N + i];

  // pass 1: H = projection of the contravariant flux (xi_x F + xi_y G, eta_x F + eta_y G)
  double Hx[4][ML], Hy[4][ML];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) { Hx[v][l] = 0.0; Hy[v][l] = 0.0; }
#pragma unroll 1
  for (int k = 0; k < NQ; ++k) {
    double q[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double acc = 0.0;
#pragma unroll
      for (int l = 0; l < ML; ++l) acc = fma(c[v][l], t.phi[k][l], acc);
      q[v] = acc;
    }
    Pt s = make_pt(g1, q[0], q[1], q[2], q[3]);
    double F[4], G[4];
    euler_flux(s, F, G);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double fx = t.w[k] * (jxx * F[v] + jxy * G[v]);
      double fy = t.w[k] * (jyx * F[v] + jyy * G[v]);
#pragma unroll
      for (int l = 0; l < ML; ++l) { Hx[v][l] = fma(fx, t.phi[k][l], Hx[v][l]); Hy[v][l] = fma(fy, t.phi[k][l], Hy[v][l]); }
    }
  }
  // pass 2: projection of the contravariant F_t
  double Tx[4][ML], Ty[4][ML];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) { Tx[v][l] = 0.0; Ty[v][l] = 0.0; }
#pragma unroll 1
  for (int k = 0; k < NQ; ++k) {
    double q[4], qt[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double acc = 0.0, dv = 0.0;
#pragma unroll
      for (int l = 0; l < ML; ++l) {
        acc = fma(c[v][l], t.phi[k][l], acc);
        dv = fma(Hx[v][l], t.dxi[k][l], dv);
        dv = fma(Hy[v][l], t.deta[k][l], dv);
      }
      q[v] = acc; qt[v] = -dv;
    }
    Pt s = make_pt(g1, q[0], q[1], q[2], q[3]);
    double F1[4], G1[4], du, dvv, dp;
    euler_d1(g1, s, qt, F1, G1, du, dvv, dp);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double fx = t.w[k] * (jxx * F1[v] + jxy * G1[v]);
      double fy = t.w[k] * (jyx * F1[v] + jyy * G1[v]);
#pragma unroll
      for (int l = 0; l < ML; ++l) { Tx[v][l] = fma(fx, t.phi[k][l], Tx[v][l]); Ty[v][l] = fma(fy, t.phi[k][l], Ty[v][l]); }
    }
  }
  // pass 2b (ORD4): projection of the contravariant F_tt
  double Ux[4][ORD4 ? ML : 1], Uy[4][ORD4 ? ML : 1];
  if (ORD4) {
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int l = 0; l < (ORD4 ? ML : 1); ++l) { Ux[v][l] = 0.0; Uy[v][l] = 0.0; }
#pragma unroll 1
    for (int k = 0; k < NQ; ++k) {
      double q[4], qt[4], qtt[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double acc = 0.0, d1 = 0.0, d2 = 0.0;
#pragma unroll
        for (int l = 0; l < ML; ++l) {
          acc = fma(c[v][l], t.phi[k][l], acc);
          d1 = fma(Hx[v][l], t.dxi[k][l], d1);
          d1 = fma(Hy[v][l], t.deta[k][l], d1);
          d2 = fma(Tx[v][l], t.dxi[k][l], d2);
          d2 = fma(Ty[v][l], t.deta[k][l], d2);
        }
        q[v] = acc; qt[v] = -d1; qtt[v] = -d2;
      }
      Pt s = make_pt(g1, q[0], q[1], q[2], q[3]);
      double F2[4], G2[4], F3[4], G3[4], du, dvv, dp, eu, ev, ep;
      double F1[4], G1[4];
      euler_d1(g1, s, qt, F1, G1, du, dvv, dp);
      euler_d2(g1, s, qt, du, dvv, dp, F2, G2);
      euler_d1(g1, s, qtt, F3, G3, eu, ev, ep);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const double Ftt = F2[v] + F3[v], Gtt = G2[v] + G3[v];
        double fx = t.w[k] * (jxx * Ftt + jxy * Gtt);
        double fy = t.w[k] * (jyx * Ftt + jyy * Gtt);
#pragma unroll
        for (int l = 0; l < (ORD4 ? ML : 1); ++l) {
          Ux[v][l] = fma(fx, t.phi[k][l], Ux[v][l]);
          Uy[v][l] = fma(fy, t.phi[k][l], Uy[v][l]);
        }
      }
    }
  }
  const double c3 = dt * dt * dt / 24.0;
  // pass 3: F_T at every point; volume integral at interior points, traces at edge points
  double Vv[4][ML];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) Vv[v][l] = 0.0;
#pragma unroll 1
  for (int p = 0; p < NPT; ++p) {
    double q[4], qt[4], qtt[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double acc = 0.0, d1 = 0.0, d2 = 0.0;
#pragma unroll
      for (int l = 0; l < ML; ++l) {
        acc = fma(c[v][l], t.phi[p][l], acc);
        d1 = fma(Hx[v][l], t.dxi[p][l], d1);
        d1 = fma(Hy[v][l], t.deta[p][l], d1);
        d2 = fma(Tx[v][l], t.dxi[p][l], d2);
        d2 = fma(Ty[v][l], t.deta[p][l], d2);
      }
      q[v] = acc; qt[v] = -d1; qtt[v] = -d2;
    }
    Pt s = make_pt(g1, q[0], q[1], q[2], q[3]);
    double F[4], G[4], F1[4], G1[4], F2[4], G2[4], F3[4], G3[4];
    double du, dvv, dp, eu, ev, ep;
    euler_flux(s, F, G);
    euler_d1(g1, s, qt, F1, G1, du, dvv, dp);
    euler_d2(g1, s, qt, du, dvv, dp, F2, G2);
    euler_d1(g1, s, qtt, F3, G3, eu, ev, ep);
    double FT[4], GT[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      FT[v] = F[v] + c1 * F1[v] + c2 * (F2[v] + F3[v]);
      GT[v] = G[v] + c1 * G1[v] + c2 * (G2[v] + G3[v]);
    }
    if (ORD4) {
      double qttt[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double d3 = 0.0;
#pragma unroll
        for (int l = 0; l < (ORD4 ? ML : 1); ++l) {
          d3 = fma(Ux[v][l], t.dxi[p][l], d3);
          d3 = fma(Uy[v][l], t.deta[p][l], d3);
        }
        qttt[v] = -d3;
      }
      double A[4], B[4], C[4], D[4], Fq[4], Gq[4], fu, fv, fp;
      euler_d3(g1, s, qt, A, B);
      euler_d11(g1, s, qt, qtt, C, D);
      euler_d1(g1, s, qttt, Fq, Gq, fu, fv, fp);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        FT[v] += c3 * (A[v] + 3.0 * C[v] + Fq[v]);
        GT[v] += c3 * (B[v] + 3.0 * D[v] + Gq[v]);
      }
    }
    if (p < NQ) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double fx = t.w[p] * (jxx * FT[v] + jxy * GT[v]);
        double fy = t.w[p] * (jyx * FT[v] + jyy * GT[v]);
#pragma unroll
        for (int l = 1; l < ML; ++l) Vv[v][l] = fma(fx, t.dxi[p][l], fma(fy, t.deta[p][l], Vv[v][l]));
      }
    } else {
      const int k = (p - NQ) / MQ, pe = (p - NQ) % MQ;
      const double nx = m.nrm[(2 * k) * N + i], ny = m.nrm[(2 * k + 1) * N + i];
      double* tr = w.trace + ((size_t)(k * MQ + pe) * 8) * N + i;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        tr[(size_t)v * N] = q[v];
        tr[(size_t)(4 + v) * N] = nx * FT[v] + ny * GT[v];
      }
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int l = 1; l < ML; ++l) Qi[v * ML + l] = c[v][l] + dt * Vv[v][l];
}

// ------------------------------------------------------------ k_edge
// Sec. 3.3 Step 3 seen from each element (the two sides of an edge compute
// bitwise-opposite values: the same operands in the same order, negated),
// the edge integral of the higher moments, and Steps 4-5 (Gamma, the
// density Lambda of the four cases, box corners and the mu quadratic).
template <int KD, int E, int ML, int NQ, int MQ>
__global__ void __launch_bounds__(128) k_edge(const DevMesh m, const DevWork w, double* __restrict__ Q,
                                              const StepArgs a) {
  const Tables& t = c_tabs[KD];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N || !step_live(a)) return;
  const int N = m.N;
  const double g = a.gamma, g1 = g - 1.0;
  const double s = __longlong_as_double((long long)*w.smax);
  const double dt = step_dt(w, m, a);
  double* Qi = Q + (size_t)i * 4 * ML;
  const double qb[4] = {Qi[0], Qi[ML], Qi[2 * ML], Qi[3 * ML]};
  const double area = m.area[i];
  double Ei[4][ML];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) Ei[v][l] = 0.0;
  double fW[E][4], fF[E][4];
  // flux of the own average, reused on every edge
  Pt sb = make_pt(g1, qb[0], qb[1], qb[2], qb[3]);
  double Fb[4], Gb[4];
  euler_flux(sb, Fb, Gb);
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int j = m.nbr[k * N + i];
    const int kj = m.nbk[k * N + i];
    const double nx = m.nrm[(2 * k) * N + i], ny = m.nrm[(2 * k + 1) * N + i];
    const double ln = sqrt(nx * nx + ny * ny);
    const double hs = 0.5 * s * ln;
    const bool owner = j < 0 || i < j || (i == j && k < kj);
    // neighbour (or exterior) average for f^LxF
    double qn[4];
    if (j >= 0) {
      const double* Qj = Q + (size_t)j * 4 * ML;
      qn[0] = Qj[0]; qn[1] = Qj[ML]; qn[2] = Qj[2 * ML]; qn[3] = Qj[3 * ML];
    } else {
      ghost_state(-1 - j, nx / ln, ny / ln, qb, qn, a.qin);
    }
    {
      Pt sn = make_pt(g1, qn[0], qn[1], qn[2], qn[3]);
      double Fn[4], Gn[4];
      euler_flux(sn, Fn, Gn);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double ai = __fma_rn(nx, Fb[v], __dmul_rn(ny, Gb[v]));
        double an = __fma_rn(nx, Fn[v], __dmul_rn(ny, Gn[v]));
        fF[k][v] = __fma_rn(-hs, __dsub_rn(qn[v], qb[v]), __dmul_rn(0.5, __dadd_rn(ai, an)));
      }
    }
    // high-order flux at the edge points, visited in the owner's order
#pragma unroll
    for (int v = 0; v < 4; ++v) fW[k][v] = 0.0;
#pragma unroll
    for (int qo = 0; qo < MQ; ++qo) {
      const int p = owner ? qo : MQ - 1 - qo;
      const double* tr = w.trace + ((size_t)(k * MQ + p) * 8) * N + i;
      double qi[4], Fi[4], qx[4], Fx[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) { qi[v] = tr[(size_t)v * N]; Fi[v] = tr[(size_t)(4 + v) * N]; }
      if (j >= 0) {
        const double* tj = w.trace + ((size_t)(kj * MQ + (MQ - 1 - p)) * 8) * N + j;
#pragma unroll
        for (int v = 0; v < 4; ++v) { qx[v] = tj[(size_t)v * N]; Fx[v] = -tj[(size_t)(4 + v) * N]; }
      } else if (-1 - j == LXW_BC_REFLECT) {
        // exterior state R q and n.F_T(R q) = -R (n.F_T(q)) (reflection symmetry of the Euler flux)
        const double nxh = nx / ln, nyh = ny / ln;
        ghost_state(LXW_BC_REFLECT, nxh, nyh, qi, qx, a.qin);
        double R[4];
        ghost_state(LXW_BC_REFLECT, nxh, nyh, Fi, R, a.qin);
#pragma unroll
        for (int v = 0; v < 4; ++v) Fx[v] = -R[v];
      } else if (-1 - j == LXW_BC_INFLOW) {
        // a steady exterior state: q_t = q_tt = 0, so F_T = F(q_in)
#pragma unroll
        for (int v = 0; v < 4; ++v) { qx[v] = a.qin[v]; Fx[v] = __fma_rn(nx, a.fin[v], __dmul_rn(ny, a.gin[v])); }
      } else {
#pragma unroll
        for (int v = 0; v < 4; ++v) { qx[v] = qi[v]; Fx[v] = Fi[v]; }
      }
      // dissipation speed: the local Lax-Friedrichs speed of the two traces,
      // at most the global s (or s itself under the literal reading)
      const double hp = a.llf_global ? hs : 0.5 * fmin(s, fmax(lf_speed(g, qi), lf_speed(g, qx))) * ln;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        // Eq. LLF scaled by the edge length
        double fs = __fma_rn(-hp, __dsub_rn(qx[v], qi[v]), __dmul_rn(0.5, __dadd_rn(Fi[v], Fx[v])));
        fW[k][v] = __fma_rn(0.5 * t.ew[qo], fs, fW[k][v]);
        const double hw = 0.5 * t.ew[p] * fs;
#pragma unroll
        for (int l = 1; l < ML; ++l) Ei[v][l] = fma(hw, t.phi[NQ + k * MQ + p][l], Ei[v][l]);
      }
    }
  }
  // higher moments: subtract the edge integral (the volume part was added by k_ck)
  const double dta = dt / area;
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int l = 1; l < ML; ++l) Qi[v * ML + l] -= dta * Ei[v][l];

  // Steps 4-5: Gamma, density Lambda, Lax-Friedrichs state, box corners, mu
  double Gam0 = area / dt * qb[0];
#pragma unroll
  for (int k = 0; k < E; ++k) Gam0 -= fF[k][0];
  if (Gam0 < 0.0) atomicOr(w.status, (unsigned)LXW_ST_CFL);
  double neg = 0.0;
#pragma unroll
  for (int k = 0; k < E; ++k) {
    double df = fF[k][0] - fW[k][0];
    if (df < 0.0) neg += df;
  }
  double ql[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < E; ++k) acc += fF[k][v];
    ql[v] = qb[v] - dta * acc;
  }
  double er = fmin(a.eps0, 0.5 * ql[0]);
  er = er > 0.0 ? er : 0.0;
  double lneg = 1.0;
  if (neg < 0.0) lneg = fmin(1.0, fmax(0.0, (Gam0 - area / dt * er) / (-neg)));
  double lam[E], dq[E][4];
#pragma unroll
  for (int k = 0; k < E; ++k) {
    lam[k] = (fF[k][0] - fW[k][0]) < 0.0 ? lneg : 1.0;
#pragma unroll
    for (int v = 0; v < 4; ++v) dq[k][v] = dta * lam[k] * (fF[k][v] - fW[k][v]);
  }
  // mu for every nonempty corner of the box [0, Lambda]
  const double pl = ql[0] > 0.0 ? g1 * (ql[3] - 0.5 * (ql[1] * ql[1] + ql[2] * ql[2]) / ql[0]) : -1.0;
  double mmin[E];
#pragma unroll
  for (int k = 0; k < E; ++k) mmin[k] = 1.0;
  if (!(ql[0] > 0.0) || !(pl > 0.0)) {
#pragma unroll
    for (int k = 0; k < E; ++k) mmin[k] = 0.0;
  } else {
    const double kap = fmin(a.eps0, 0.5 * pl) / g1;
    const double h0 = ql[0] * ql[3] - 0.5 * (ql[1] * ql[1] + ql[2] * ql[2]) - kap * ql[0];
#pragma unroll
    for (int cm = 1; cm < (1 << E); ++cm) {
      double d[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 0; k < E; ++k)
        if ((cm >> k) & 1)
#pragma unroll
          for (int v = 0; v < 4; ++v) d[v] += dq[k][v];
      // h(mu) = rho E - |M|^2/2 - kappa rho along ql + mu d
      const double h1 = ql[0] * d[3] + d[0] * ql[3] - (ql[1] * d[1] + ql[2] * d[2]) - kap * d[0];
      const double h2 = d[0] * d[3] - 0.5 * (d[1] * d[1] + d[2] * d[2]);
      double mu = 1.0;
      if (!(ql[0] + d[0] > 0.0) || h0 + h1 + h2 < 0.0) {
        double disc = fmax(h1 * h1 - 4.0 * h0 * h2, 0.0);
        double den = -h1 + sqrt(disc);
        mu = den > 0.0 ? fmin(1.0, fmax(0.0, 2.0 * h0 / den)) : 0.0;
      }
#pragma unroll
      for (int k = 0; k < E; ++k)
        if ((cm >> k) & 1) mmin[k] = fmin(mmin[k], mu);
    }
  }
#pragma unroll
  for (int k = 0; k < E; ++k) {
    w.prop[k * N + i] = lam[k] * mmin[k];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      w.flux[(size_t)(k * 8 + v) * N + i] = fW[k][v];
      w.flux[(size_t)(k * 8 + 4 + v) * N + i] = fF[k][v];
    }
  }
}

// ------------------------------------------------------------ k_update
// Sec. 3.3 Step 6: theta_k = min of the two sides' proposals; blended
// update of the cell averages.
template <int E, int ML>
__global__ void __launch_bounds__(128) k_update(const DevMesh m, const DevWork w, double* __restrict__ Q, const StepArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N || !step_live(a)) return;
  const int N = m.N;
  const double dt = step_dt(w, m, a);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int j = m.nbr[k * N + i];
    double th = w.prop[k * N + i];
    if (j >= 0) th = fmin(th, w.prop[m.nbk[k * N + i] * N + j]);
    if (a.theta_edge) a.theta_edge[(size_t)i * E + k] = th;
    if (a.want_diag && th < 1.0 && (j < 0 || i < j || (i == j && k < m.nbk[k * N + i])))
      atomicAdd(&reinterpret_cast<DevDiag*>(w.diag)->nedge, 1ull);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double fw = w.flux[(size_t)(k * 8 + v) * N + i], ff = w.flux[(size_t)(k * 8 + 4 + v) * N + i];
      acc[v] += th * fw + (1.0 - th) * ff;
    }
  }
  double* Qi = Q + (size_t)i * 4 * ML;
  const double dta = dt / m.area[i];
#pragma unroll
  for (int v = 0; v < 4; ++v) Qi[v * ML] -= dta * acc[v];
}

// ------------------------------------------------------------ k_shock
// Sec. 4.1 shock-capturing limiter on the primitive variables (rho,u,v,p):
// M = max(w_i + alpha, max_j w_j), m = min(w_i - alpha, min_j w_j) over the
// face neighbours, theta = min(1, (M - w_i)/(max_pts - w_i), (w_i - m)/(w_i - min_pts)).
template <int KD, int E, int ML, int NQ, int MQ>
__global__ void __launch_bounds__(128) k_shock(const DevMesh m, double* __restrict__ Q, const StepArgs a,
                                               double* __restrict__ theta_out, unsigned long long* nsc) {
  constexpr int NPT = NQ + E * MQ;
  const Tables& t = c_tabs[KD];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N || !step_live(a)) return;
  const int N = m.N;
  const double g1 = a.gamma - 1.0;
  double* Qi = Q + (size_t)i * 4 * ML;
  double c[4][ML];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) c[v][l] = Qi[v * ML + l];
  double th = 1.0;
  if (!(c[0][0] > 0.0)) {
    th = 0.0;
  } else {
    Pt sb = make_pt(g1, c[0][0], c[1][0], c[2][0], c[3][0]);
    const double wb[4] = {sb.r, sb.u, sb.v, sb.p};
    const double dx = m.sdx[i];
    const double al = a.alpha0 * dx * sqrt(dx);
    double Mx[4], Mn[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) { Mx[v] = wb[v] + al; Mn[v] = wb[v] - al; }
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int j = m.nbr[k * N + i];
      double qn[4];
      if (j >= 0) {
        const double* Qj = Q + (size_t)j * 4 * ML;
        qn[0] = Qj[0]; qn[1] = Qj[ML]; qn[2] = Qj[2 * ML]; qn[3] = Qj[3 * ML];
      } else {
        const double nx = m.nrm[(2 * k) * N + i], ny = m.nrm[(2 * k + 1) * N + i];
        const double ln = sqrt(nx * nx + ny * ny);
        const double qbv[4] = {c[0][0], c[1][0], c[2][0], c[3][0]};
        ghost_state(-1 - j, nx / ln, ny / ln, qbv, qn, a.qin);
      }
      if (!(qn[0] > 0.0)) continue;
      Pt sn = make_pt(g1, qn[0], qn[1], qn[2], qn[3]);
      const double wn[4] = {sn.r, sn.u, sn.v, sn.p};
#pragma unroll
      for (int v = 0; v < 4; ++v) { Mx[v] = fmax(Mx[v], wn[v]); Mn[v] = fmin(Mn[v], wn[v]); }
    }
    double hx[4], hn[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) { hx[v] = -1e300; hn[v] = 1e300; }
    bool bad = false;
#pragma unroll
    for (int p = 0; p < NPT; ++p) {
      double q[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double acc = 0.0;
#pragma unroll
        for (int l = 0; l < ML; ++l) acc = fma(c[v][l], t.phi[p][l], acc);
        q[v] = acc;
      }
      if (!(q[0] > 0.0)) { bad = true; break; }
      Pt sp = make_pt(g1, q[0], q[1], q[2], q[3]);
      const double wp[4] = {sp.r, sp.u, sp.v, sp.p};
#pragma unroll
      for (int v = 0; v < 4; ++v) { hx[v] = fmax(hx[v], wp[v]); hn[v] = fmin(hn[v], wp[v]); }
    }
    if (bad) {
      th = 0.0;
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        if (hx[v] > wb[v]) th = fmin(th, (Mx[v] - wb[v]) / (hx[v] - wb[v]));
        if (hn[v] < wb[v]) th = fmin(th, (wb[v] - Mn[v]) / (wb[v] - hn[v]));
      }
      th = fmax(th, 0.0);
    }
  }
  if (th < 1.0) {
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int l = 1; l < ML; ++l) Qi[v * ML + l] = th * c[v][l];
    if (nsc) atomicAdd(nsc, 1ull);
  }
  if (theta_out) theta_out[i] = th;
}

// ------------------------------------------------------------ k_diag
template <int ML>
__global__ void __launch_bounds__(256) k_diag(const DevMesh m, const DevWork w, const double* __restrict__ Q, double gamma) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  DevDiag* d = reinterpret_cast<DevDiag*>(w.diag);
  if (i < m.N) {
    const double* Qi = Q + (size_t)i * 4 * ML;
    double q[4] = {Qi[0], Qi[ML], Qi[2 * ML], Qi[3 * ML]};
    double p = (gamma - 1.0) * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / q[0]);
    bool finite = true;
    for (int v = 0; v < 4; ++v) finite = finite && isfinite(q[v]);
    if (!finite) atomicOr(w.status, (unsigned)LXW_ST_NAN);
    const double a = m.area[i];
    for (int v = 0; v < 4; ++v) atomicAdd(&d->sum[v], a * q[v]);
    atomicMin(&d->minr, ordered_bits(q[0]));
    atomicMin(&d->minp, ordered_bits(p));
  }
}

// ------------------------------------------------------------ k_project
// Initial-condition L2 projection Q^(l) = sum_p w_p q(x_p) phi_l(x_p).
__global__ void k_project(const ProjTables t, int N, double gamma, const double* __restrict__ prim,
                          double* __restrict__ Q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double acc[4][kMaxML];
  for (int v = 0; v < 4; ++v)
    for (int l = 0; l < t.ML; ++l) acc[v][l] = 0.0;
  for (int p = 0; p < t.NPJ; ++p) {
    const double* w = prim + ((size_t)i * t.NPJ + p) * 4;
    double q[4] = {w[0], w[0] * w[1], w[0] * w[2], w[3] / (gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2])};
    for (int v = 0; v < 4; ++v)
      for (int l = 0; l < t.ML; ++l) acc[v][l] += t.w[p] * q[v] * t.phi[p][l];
  }
  for (int v = 0; v < 4; ++v)
    for (int l = 0; l < t.ML; ++l) Q[((size_t)i * 4 + v) * t.ML + l] = acc[v][l];
}

__global__ void k_copy_speed(DevWork w, double* s_dev) {
  *s_dev = __longlong_as_double((long long)*w.smax);
}

inline int grid_for(int N, int block) { return (N + block - 1) / block; }

template <int KD, int E, int ML, int NQ, int MQ>
int step_impl(const DevMesh& m, const DevWork& w, double* Q, const StepArgs& a, cudaStream_t st, int block,
              void** events, int upto) {
  const int grid = grid_for(m.N, block);
  DevDiag* dd = reinterpret_cast<DevDiag*>(w.diag);
  int ne = 0;
  auto mark = [&]() { if (events) cudaEventRecordWithFlags((cudaEvent_t)events[ne++], st, cudaEventRecordExternal); };
  mark();
  k_reset<<<1, 1, 0, st>>>(w, a.want_diag, 0);   // status bits stay until a diagnostic step reads them
  mark();
  if (a.moment_exact)
    k_moment<KD, E, ML, NQ, MQ, true><<<grid, block, 0, st>>>(m, w, Q, a, a.theta_cell);
  else
    k_moment<KD, E, ML, NQ, MQ><<<grid, block, 0, st>>>(m, w, Q, a, a.theta_cell);
  mark();
  if (upto < 2) return cudaGetLastError() == cudaSuccess ? 0 : -1;
  if (a.ck_order == 4)
    k_ck<KD, E, ML, NQ, MQ, true><<<grid, block, 0, st>>>(m, w, Q, a);
  else
    k_ck<KD, E, ML, NQ, MQ><<<grid, block, 0, st>>>(m, w, Q, a);
  mark();
  if (upto < 3) return cudaGetLastError() == cudaSuccess ? 0 : -1;
  k_edge<KD, E, ML, NQ, MQ><<<grid, block, 0, st>>>(m, w, Q, a);
  mark();
  if (upto < 4) return cudaGetLastError() == cudaSuccess ? 0 : -1;
  k_update<E, ML><<<grid, block, 0, st>>>(m, w, Q, a);
  mark();
  if (a.shock_limiter && upto >= 5) {
    k_shock<KD, E, ML, NQ, MQ><<<grid, block, 0, st>>>(m, Q, a, a.theta_cell ? a.theta_cell + m.N : nullptr,
                                                       a.want_diag ? &dd->nsc : nullptr);
    mark();
  }
  if (a.timed) k_clock<<<1, 1, 0, st>>>(m, w, a);
  if (a.want_diag) k_diag<ML><<<grid_for(m.N, 256), 256, 0, st>>>(m, w, Q, a.gamma);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int KD, int E, int ML, int NQ, int MQ>
int moment_impl(const DevMesh& m, const DevWork& w, double* Q, const StepArgs& a, double* theta,
                cudaStream_t st, int block) {
  k_reset<<<1, 1, 0, st>>>(w, 0, 1);
  if (a.moment_exact)
    k_moment<KD, E, ML, NQ, MQ, true><<<grid_for(m.N, block), block, 0, st>>>(m, w, Q, a, theta);
  else
    k_moment<KD, E, ML, NQ, MQ><<<grid_for(m.N, block), block, 0, st>>>(m, w, Q, a, theta);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int KD, int E, int ML, int NQ, int MQ>
int shock_impl(const DevMesh& m, double* Q, const StepArgs& a, double* theta, cudaStream_t st, int block) {
  k_shock<KD, E, ML, NQ, MQ><<<grid_for(m.N, block), block, 0, st>>>(m, Q, a, theta, nullptr);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

#define LXW_DISPATCH(kind, deg, CALL)                                   \
  do {                                                                  \
    if (kind == LXW_KIND_QUAD && deg == 2) return CALL(0, 4, 6, 9, 3);   \
    if (kind == LXW_KIND_QUAD && deg == 3) return CALL(1, 4, 10, 16, 4); \
    if (kind == LXW_KIND_TRI && deg == 2) return CALL(2, 3, 6, 9, 3);    \
    if (kind == LXW_KIND_TRI && deg == 3) return CALL(3, 3, 10, 16, 4);  \
    return -2;                                                          \
  } while (0)

int launch_step(int kind, int deg, const DevMesh& m, const DevWork& w, double* Q, const StepArgs& a,
                void* stream, int block, void** events, int upto) {
#define CALL_STEP(KD, E, ML, NQ, MQ) \
  step_impl<KD, E, ML, NQ, MQ>(m, w, Q, a, (cudaStream_t)stream, block, events, upto)
  LXW_DISPATCH(kind, deg, CALL_STEP);
#undef CALL_STEP
}

int launch_moment_limit(int kind, int deg, const DevMesh& m, const DevWork& w, double* Q,
                        const StepArgs& a, double* theta, void* stream, int block) {
#define CALL_MOM(KD, E, ML, NQ, MQ) moment_impl<KD, E, ML, NQ, MQ>(m, w, Q, a, theta, (cudaStream_t)stream, block)
  LXW_DISPATCH(kind, deg, CALL_MOM);
#undef CALL_MOM
}

int launch_shock_limit(int kind, int deg, const DevMesh& m, double* Q, const StepArgs& a,
                       double* theta, void* stream, int block) {
#define CALL_SH(KD, E, ML, NQ, MQ) shock_impl<KD, E, ML, NQ, MQ>(m, Q, a, theta, (cudaStream_t)stream, block)
  LXW_DISPATCH(kind, deg, CALL_SH);
#undef CALL_SH
}

int launch_project(const ProjTables& t, int N, double gamma, const double* prim, double* Q, void* stream) {
  k_project<<<grid_for(N, 128), 128, 0, (cudaStream_t)stream>>>(t, N, gamma, prim, Q);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_copy_speed(const DevWork& w, double* s_dev, void* stream) {
  k_copy_speed<<<1, 1, 0, (cudaStream_t)stream>>>(w, s_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int upload_tables(int kind, int deg, const Tables& t) {
  const int kd = (kind == LXW_KIND_QUAD ? 0 : 2) + (deg == 3 ? 1 : 0);
  return cudaMemcpyToSymbol(c_tabs, &t, sizeof(Tables), kd * sizeof(Tables)) == cudaSuccess ? 0 : -1;
}

int step_launch_count(int want_diag, int shock_limiter) { return 5 + (shock_limiter ? 1 : 0) + (want_diag ? 1 : 0); }

// host-side decoding of the diagnostics block
void decode_diag(const double* raw, double out[9]) {
  const DevDiag* d = reinterpret_cast<const DevDiag*>(raw);
  unsigned long long b;
  for (int v = 0; v < 4; ++v) out[v] = d->sum[v];
  b = d->minr; b = (b & 0x8000000000000000ull) ? (b & 0x7fffffffffffffffull) : ~b;
  double x; memcpy(&x, &b, 8); out[4] = x;
  b = d->minp; b = (b & 0x8000000000000000ull) ? (b & 0x7fffffffffffffffull) : ~b;
  memcpy(&x, &b, 8); out[5] = x;
  out[6] = (double)d->nmom; out[7] = (double)d->nedge; out[8] = (double)d->nsc;
}
size_t diag_bytes() { return sizeof(DevDiag); }

}  // namespace lxw

// ====================================================================
// Allocation-free variant of the moment limiter and wave-speed reduction.
//
// Some callers cannot call cudaMalloc: code whose device memory belongs to
// another allocator (a framework's caching pool, or a fixed budget carved
// out at start-up, where a stray allocation could fail or fragment it), and
// code that must not take cudaMalloc's implicit device synchronisation (a
// time-critical loop sharing the GPU with other streams).
// lxw_moment_limit_noalloc serves them: it needs no solver (whose creation
// allocates), only the caller's state, theta and speed buffers.  The
// reduction scratch of the wave speed -- one running maximum per chunk of
// kNoAllocChunk elements and a status word -- lives in the file-scope array
// below, which every GPU that loads the library holds until exit.
// ====================================================================
#include <mutex>
#include <string>

namespace lxw {
namespace {

constexpr int kNoAllocChunk = 32768;          // elements per reduction slot
constexpr int kNoAllocSlots = 512;            // -> at most 16,777,216 elements
constexpr int kMaxDevices = 64;

// slot maxima (bits of non-negative doubles), then one status word
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocSlots + 1];

// zero the slots this call uses and the status word
__global__ void k_noalloc_clear(int nslots) {
  for (int c = threadIdx.x; c < nslots; c += blockDim.x) g_noalloc_scratch[c] = 0ull;
  if (threadIdx.x == 0) g_noalloc_scratch[kNoAllocSlots] = 0ull;
}

__global__ void k_noalloc_finish(int nslots, double* s_dev, unsigned int* status_dev) {
  unsigned long long m = 0ull;
  for (int c = 0; c < nslots; ++c) m = m > g_noalloc_scratch[c] ? m : g_noalloc_scratch[c];
  *s_dev = __longlong_as_double((long long)m);
  if (status_dev) *status_dev = (unsigned int)g_noalloc_scratch[kNoAllocSlots];
}

std::mutex g_noalloc_mu;
unsigned long long* g_noalloc_addr[kMaxDevices] = {};
bool g_noalloc_tables[kMaxDevices][4] = {};

template <int KD, int E, int ML, int NQ, int MQ>
void noalloc_impl(int N, double* Q, const StepArgs& a, double* theta, double* s_dev, unsigned int* status_dev,
                  cudaStream_t st, unsigned long long* scratch) {
  const int nslots = (N + kNoAllocChunk - 1) / kNoAllocChunk;
  k_noalloc_clear<<<1, 256, 0, st>>>(nslots);
  for (int c = 0; c < nslots; ++c) {
    const int n = N - c * kNoAllocChunk < kNoAllocChunk ? N - c * kNoAllocChunk : kNoAllocChunk;
    DevMesh m{};
    m.N = n;                                   // the moment kernel reads only N
    DevWork w{};
    w.smax = scratch + c;
    w.status = reinterpret_cast<unsigned int*>(scratch + kNoAllocSlots);
    k_moment<KD, E, ML, NQ, MQ><<<grid_for(n, 128), 128, 0, st>>>(
        m, w, Q + (size_t)c * kNoAllocChunk * 4 * ML, a, theta ? theta + (size_t)c * kNoAllocChunk : nullptr);
  }
  k_noalloc_finish<<<1, 1, 0, st>>>(nslots, s_dev, status_dev);
}

}  // namespace
}  // namespace lxw

extern "C" lxw_status lxw_moment_limit_noalloc(int kind, int degree, int n_elements, double gamma, double eps0,
                                               double* Q_dev, double* theta_dev, double* s_dev,
                                               unsigned int* status_dev, void* stream) {
  using namespace lxw;
  auto err = [](lxw_status st, const char* msg) { set_last_error(msg); return st; };
  auto cuda_err = [](const char* what, cudaError_t e) {
    std::string m = std::string("lxw_moment_limit_noalloc: ") + what + ": " + cudaGetErrorString(e);
    set_last_error(m.c_str());
    return LXW_ERR_CUDA;
  };
  // an error left by earlier work on this thread belongs to that work: report
  // it without clearing it, and launch nothing
  if (cudaError_t e = cudaPeekAtLastError(); e != cudaSuccess) return cuda_err("a CUDA error was already pending", e);
  if (!Q_dev || !s_dev) return err(LXW_ERR_ARG, "lxw_moment_limit_noalloc: null Q_dev or s_dev");
  if ((kind != LXW_KIND_QUAD && kind != LXW_KIND_TRI) || (degree != 2 && degree != 3))
    return err(LXW_ERR_ARG, "lxw_moment_limit_noalloc: kind must be quad/triangle and degree 2 or 3");
  if (n_elements < 1 || n_elements > kNoAllocChunk * kNoAllocSlots)
    return err(LXW_ERR_ARG, "lxw_moment_limit_noalloc: n_elements must be in [1, 16777216] (static scratch capacity)");
  if (!(gamma > 1.0) || !(eps0 > 0.0)) return err(LXW_ERR_ARG, "lxw_moment_limit_noalloc: need gamma > 1 and eps0 > 0");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return err(LXW_ERR_CUDA, "lxw_moment_limit_noalloc: no usable current device");
  const int kd = (kind == LXW_KIND_QUAD ? 0 : 2) + (degree == 3 ? 1 : 0);
  unsigned long long* scratch = nullptr;
  {
    // once per device (with that device current): the device address of the
    // scratch array and this variant's tables in the constant bank
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
        return err(LXW_ERR_CUDA, "lxw_moment_limit_noalloc: cudaGetSymbolAddress of the scratch array failed");
      g_noalloc_addr[dev] = static_cast<unsigned long long*>(p);
    }
    if (!g_noalloc_tables[dev][kd]) {
      Tables t;
      make_tables(kind, degree, t);
      if (upload_tables(kind, degree, t)) return err(LXW_ERR_CUDA, "lxw_moment_limit_noalloc: table upload failed");
      g_noalloc_tables[dev][kd] = true;
    }
    scratch = g_noalloc_addr[dev];
  }
  StepArgs a{};
  a.gamma = gamma;
  a.eps0 = eps0;
  cudaStream_t st = (cudaStream_t)stream;
  if (kd == 0) noalloc_impl<0, 4, 6, 9, 3>(n_elements, Q_dev, a, theta_dev, s_dev, status_dev, st, scratch);
  else if (kd == 1) noalloc_impl<1, 4, 10, 16, 4>(n_elements, Q_dev, a, theta_dev, s_dev, status_dev, st, scratch);
  else if (kd == 2) noalloc_impl<2, 3, 6, 9, 3>(n_elements, Q_dev, a, theta_dev, s_dev, status_dev, st, scratch);
  else noalloc_impl<3, 3, 10, 16, 4>(n_elements, Q_dev, a, theta_dev, s_dev, status_dev, st, scratch);
  if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return cuda_err("launch failed", e);
  if (status_dev) return LXW_OK;
  // no status pointer: wait for the call and read the status word (into a
  // host variable: no allocation)
  unsigned int word = 0;
  if (cudaError_t e = cudaMemcpyFromSymbolAsync(&word, g_noalloc_scratch, sizeof(word),
                                                 kNoAllocSlots * sizeof(unsigned long long),
                                                 cudaMemcpyDeviceToHost, st);
      e != cudaSuccess)
    return cuda_err("reading the status word failed", e);
  if (cudaError_t e = cudaStreamSynchronize(st); e != cudaSuccess) return cuda_err("waiting for the stream failed", e);
  if (word & LXW_ST_NONPOSITIVE)
    return err(LXW_ERR_NONPOSITIVE,
               "lxw_moment_limit_noalloc: an input cell average had rho <= 0 or p <= 0 (its higher modes were zeroed)");
  return LXW_OK;
}
