// lxw_kernels_mx.cu -- mixed-precision form of the LxW-DG step for sm_103a.
//
// GB300 runs FP32 fused multiply-adds ~60x faster than FP64 ones, so the
// bulk of the step -- point values, the CK time-averaged flux, the
// projections, the LLF point fluxes, volume and edge integrals -- runs in
// FP32 with FP32 higher modes and traces.  FP64 stays where the positivity
// guarantee lives (Sec. 3): the cell averages and their blended update
// (Step 6), the Lax-Friedrichs fluxes that enter that update, the Gamma /
// Lambda / box-corner / mu solve of the flux limiter (Steps 4-5) and the
// moment limiter's theta (Sec. 3.1).  Those FP64 solves run only where an
// FP32 screen with an explicit error margin cannot show that the exact
// answer is theta = 1 (no limiting); where it can, the FP64 computation
// would return exactly 1 and is skipped.
//
// State layout: averages double [4][N], their FP32 copy float [4][N] (kept
// in step with the doubles so the FP32 kernels never convert), then higher
// modes float [4][ML-1][N] (structure of arrays: a warp's loads of one
// coefficient are coalesced).  On GB300 every FP64-pipe instruction --
// DFMA, DADD, DSETP, double<->float conversion, the DDIV sequence -- runs at
// the FP64 rate, so the FP32 kernels use FP32 geometry copies and per-step
// scalars computed once per step (by the last CTA of the moment kernel) and
// touch no double at all unless a screen sends a cell to its FP64 path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "lxw_internal.h"

namespace lxw {
namespace {

struct TablesF {
  float w[kMaxQ];
  float ew[kMaxMQ];
  float phi[kMaxPts][kMaxML];
  float dxi[kMaxPts][kMaxML];
  float deta[kMaxPts][kMaxML];
};
__constant__ TablesF c_tabf[4];
// weighted differentiation tables (DerivTables, FP32)
__constant__ float c_wd[4][2][kMaxQ][kMaxML];
// the basis at the limiter points in FP64, for the moment limiter's FP64 path
// (an FP32 table promoted to double would put 1e-7 into point values whose
// pressure the secant then divides by near vacuum)
__constant__ double c_phid[4][kMaxPts][kMaxML];
// max over the limiter points of |phi_l|: the moment screen's per-cell bound
// of the point values' magnitude sums
__constant__ float c_phimax[4][kMaxML];

constexpr float kTol = 1e-5f;            // relative margin of the FP32 screens (FP32 error ~5e-7)
constexpr float kSpeedInflate = 1.00001f; // s from FP32 point values, inflated to bound the exact one

// ----------------------------------------------------------- FP32 physics
struct PtF {
  float r, m, n, e, ri, u, v, p;
};
__device__ __forceinline__ PtF ptf(float g1, float r, float m, float n, float e) {
  PtF s;
  s.r = r; s.m = m; s.n = n; s.e = e;
  s.ri = 1.0f / r;
  s.u = m * s.ri; s.v = n * s.ri;
  s.p = g1 * (e - 0.5f * (m * s.u + n * s.v));
  return s;
}
__device__ __forceinline__ void fluxf(const PtF& s, float F[4], float G[4]) {
  float h = s.e + s.p;
  F[0] = s.m; F[1] = s.m * s.u + s.p; F[2] = s.m * s.v; F[3] = h * s.u;
  G[0] = s.n; G[1] = s.n * s.u; G[2] = s.n * s.v + s.p; G[3] = h * s.v;
}
__device__ __forceinline__ void d1f(float g1, const PtF& s, const float w[4], float F[4], float G[4], float& du,
                                    float& dv, float& dp) {
  du = (w[1] - s.u * w[0]) * s.ri;
  dv = (w[2] - s.v * w[0]) * s.ri;
  float dK = s.u * w[1] + s.v * w[2] - 0.5f * (s.u * s.u + s.v * s.v) * w[0];
  dp = g1 * (w[3] - dK);
  float h = s.e + s.p, dh = w[3] + dp;
  F[0] = w[1]; F[1] = w[1] * s.u + s.m * du + dp; F[2] = w[1] * s.v + s.m * dv; F[3] = dh * s.u + h * du;
  G[0] = w[2]; G[1] = w[2] * s.u + s.n * du; G[2] = w[2] * s.v + s.n * dv + dp; G[3] = dh * s.v + h * dv;
}
__device__ __forceinline__ void d2f(float g1, const PtF& s, const float w[4], float du, float dv, float dp,
                                    float F[4], float G[4]) {
  float ddu = -2.0f * du * w[0] * s.ri, ddv = -2.0f * dv * w[0] * s.ri;
  float ddp = -g1 * s.r * (du * du + dv * dv);
  float h = s.e + s.p, dh = w[3] + dp;
  F[0] = 0.0f; F[1] = 2.0f * w[1] * du + s.m * ddu + ddp; F[2] = 2.0f * w[1] * dv + s.m * ddv;
  F[3] = ddp * s.u + 2.0f * dh * du + h * ddu;
  G[0] = 0.0f; G[1] = 2.0f * w[2] * du + s.n * ddu; G[2] = 2.0f * w[2] * dv + s.n * ddv + ddp;
  G[3] = ddp * s.v + 2.0f * dh * dv + h * ddv;
}
// third derivative of (F, G) along w and the mixed second derivative, for
// the fourth-order time average (see the FP64 kernels)
__device__ __forceinline__ void d3f(float g1, const PtF& s, const float w[4], float F[4], float G[4]) {
  const float u1 = (w[1] - s.u * w[0]) * s.ri, v1 = (w[2] - s.v * w[0]) * s.ri;
  const float u2 = -w[0] * u1 * s.ri, v2 = -w[0] * v1 * s.ri;
  const float u3 = -w[0] * u2 * s.ri, v3 = -w[0] * v2 * s.ri;
  const float p3 = -g1 * 0.5f * (s.m * u3 + w[1] * u2 + s.n * v3 + w[2] * v2);
  const float K2 = 0.5f * (s.m * u2 + w[1] * u1 + s.n * v2 + w[2] * v1);
  const float K1 = 0.5f * (s.m * u1 + w[1] * s.u + s.n * v1 + w[2] * s.v);
  const float p2 = -g1 * K2, p1 = g1 * (w[3] - K1);
  const float H0 = s.e + s.p, H1 = w[3] + p1;
  F[0] = 0.0f;
  F[1] = 6.0f * (s.m * u3 + w[1] * u2 + p3);
  F[2] = 6.0f * (s.m * v3 + w[1] * v2);
  F[3] = 6.0f * (H0 * u3 + H1 * u2 + p2 * u1 + p3 * s.u);
  G[0] = 0.0f;
  G[1] = 6.0f * (s.n * u3 + w[2] * u2);
  G[2] = 6.0f * (s.n * v3 + w[2] * v2 + p3);
  G[3] = 6.0f * (H0 * v3 + H1 * v2 + p2 * v1 + p3 * s.v);
}
__device__ __forceinline__ void d11f(float g1, const PtF& s, const float a[4], const float b[4], float F[4],
                                     float G[4]) {
  const float ua = (a[1] - s.u * a[0]) * s.ri, va = (a[2] - s.v * a[0]) * s.ri;
  const float ub = (b[1] - s.u * b[0]) * s.ri, vb = (b[2] - s.v * b[0]) * s.ri;
  const float uab = -(ub * a[0] + ua * b[0]) * s.ri, vab = -(vb * a[0] + va * b[0]) * s.ri;
  const float pa = g1 * (a[3] - (s.u * a[1] + s.v * a[2] - 0.5f * (s.u * s.u + s.v * s.v) * a[0]));
  const float pb = g1 * (b[3] - (s.u * b[1] + s.v * b[2] - 0.5f * (s.u * s.u + s.v * s.v) * b[0]));
  const float pab = -g1 * s.r * (ua * ub + va * vb);
  const float H = s.e + s.p, Ha = a[3] + pa, Hb = b[3] + pb;
  F[0] = 0.0f;
  F[1] = a[1] * ub + b[1] * ua + s.m * uab + pab;
  F[2] = a[1] * vb + b[1] * va + s.m * vab;
  F[3] = pab * s.u + Ha * ub + Hb * ua + H * uab;
  G[0] = 0.0f;
  G[1] = a[2] * ub + b[2] * ua + s.n * uab;
  G[2] = a[2] * vb + b[2] * va + s.n * vab + pab;
  G[3] = pab * s.v + Ha * vb + Hb * va + H * vab;
}
__device__ __forceinline__ float speedf(float g, float r, float m, float n, float e) {
  float ri = 1.0f / r, k2 = m * m + n * n;
  float p = (g - 1.0f) * (e - 0.5f * k2 * ri);
  p = p > 0.0f ? p : 0.0f;
  return sqrtf(k2) * ri + sqrtf(g * p * ri);
}
// exterior state of a boundary face: reflective, transparent (Sec. 2.4) or
// the prescribed inflow state qin
// |u| + c of a point state for the dissipation of the LLF point flux: both
// elements of an edge evaluate it on the same two traces and must get the
// same value (their fluxes are exact negatives), so every operation is
// pinned: the multiplies and adds explicitly rounded, the reciprocal square
// root and the square roots the hardware's approximations (deterministic;
// a few ulp, far inside the FP32 budget of a dissipation coefficient).  A
// non-positive density gives NaN, which the fminf / fmaxf that combine the
// speeds discard.
__device__ __forceinline__ float lf_speedf(float g, const float q[4]) {
  float rs, sk, sp;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(q[0]));
  const float ri = __fmul_rn(rs, rs);
  const float kin2 = __fmaf_rn(q[1], q[1], __fmul_rn(q[2], q[2]));
  float p = __fmul_rn(g - 1.0f, __fmaf_rn(__fmul_rn(-0.5f, kin2), ri, q[3]));
  p = p > 0.0f ? p : 0.0f;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sk) : "f"(kin2));
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sp) : "f"(__fmul_rn(g, p)));
  return __fmaf_rn(sk, ri, __fmul_rn(sp, rs));
}

template <typename T>
__device__ __forceinline__ void ghostq(int bc, T nxh, T nyh, const T qi[4], T qo[4], const T qin[4]) {
  if (bc == LXW_BC_INFLOW) {
#pragma unroll
    for (int v = 0; v < 4; ++v) qo[v] = qin[v];
    return;
  }
  qo[0] = qi[0]; qo[3] = qi[3];
  if (bc == LXW_BC_REFLECT) {
    T mn = qi[1] * nxh + qi[2] * nyh;
    qo[1] = qi[1] - T(2) * mn * nxh;
    qo[2] = qi[2] - T(2) * mn * nyh;
  } else {
    qo[1] = qi[1]; qo[2] = qi[2];
  }
}

// ----------------------------------------------------------- FP64 helpers
// Largest theta in [0, thr] keeping p >= ep at a point whose limited state is
// q(theta) = qbar + theta d (Sec. 3.1: the optimal theta computed exactly).
// h(theta) = (rho p - ep rho)/(g-1) = h0 + h1 theta + h2 theta^2 is positive
// at 0 and negative at thr when it is called: its one root there, in the
// cancellation-free form.
__device__ __forceinline__ double exact_root_theta(double rb, double mb, double nb, double eb, const double d[4],
                                                   double kappa, double thr) {
  const double h0 = rb * eb - 0.5 * (mb * mb + nb * nb) - kappa * rb;
  const double h1 = rb * d[3] + d[0] * eb - (mb * d[1] + nb * d[2]) - kappa * d[0];
  const double h2 = d[0] * d[3] - 0.5 * (d[1] * d[1] + d[2] * d[2]);
  const double disc = fmax(h1 * h1 - 4.0 * h0 * h2, 0.0);
  const double den = -h1 + sqrt(disc);
  return den > 0.0 ? fmin(2.0 * h0 / den, thr) : 0.0;
}

__device__ __forceinline__ void flux64(double g1, const double q[4], double F[4], double G[4]) {
  double ri = 1.0 / q[0];
  double u = q[1] * ri, v = q[2] * ri;
  double p = g1 * (q[3] - 0.5 * (q[1] * u + q[2] * v));
  double h = q[3] + p;
  F[0] = q[1]; F[1] = q[1] * u + p; F[2] = q[1] * v; F[3] = h * u;
  G[0] = q[2]; G[1] = q[2] * u; G[2] = q[2] * v + p; G[3] = h * v;
}
// Lax-Friedrichs edge flux from two averages (Sec. 3.2), outward for the
// element owning qi.  The two sides of an edge call it with (n, qi, qj) and
// (-n, qj, qi) and get exact negatives.
__device__ __forceinline__ void lxf64(double g1, double s, double nx, double ny, const double qi[4],
                                      const double qj[4], double f[4]) {
  double Fi[4], Gi[4], Fj[4], Gj[4];
  flux64(g1, qi, Fi, Gi);
  flux64(g1, qj, Fj, Gj);
  const double hs = 0.5 * s * sqrt(nx * nx + ny * ny);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    double ai = __fma_rn(nx, Fi[v], __dmul_rn(ny, Gi[v]));
    double aj = __fma_rn(nx, Fj[v], __dmul_rn(ny, Gj[v]));
    f[v] = __fma_rn(-hs, __dsub_rn(qj[v], qi[v]), __dmul_rn(0.5, __dadd_rn(ai, aj)));
  }
}

__device__ __forceinline__ unsigned long long obits(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

// per problem (one thread each): the step's wave speed and time step, in FP64 and FP32
// a problem's wave speed and time step from its running maximum (Sec. 3.2 s,
// the CFL rule), with the FP32 copies the bulk kernels use
// the CFL rule, the last step of a timed run shortened to land on t_end and
// the problem's clock advanced (once a problem's clock has reached t_end its
// kernels skip it: live = 0, the last step's s and dt kept)
__device__ __forceinline__ ScalMx make_scal(const DevMesh& m, const DevWorkMx& w, const StepArgs& a, int p) {
  const double s = __longlong_as_double((long long)__ldcg(w.smax + p));
  double dt = a.dt_in > 0.0 ? a.dt_in : a.cfl * m.hmin_p[p] / s;
  ScalMx sc;
  if (a.timed) {
    double* tc = a.tclock + 4 * p;
    const double t = tc[0];
    if (!(t < a.t_end)) {
      sc = w.scal[p];
      sc.live = 0;
      return sc;
    }
    const bool last = t + dt >= a.t_end;
    if (last) dt = a.t_end - t;
    tc[0] = last ? a.t_end : t + dt;
    tc[1] += 1.0;
    tc[2] = dt;
    tc[3] = s;
  }
  sc.s = s; sc.dt = dt;
  sc.s32 = (float)s; sc.dt32 = (float)dt; sc.c1 = (float)(0.5 * dt); sc.c2 = (float)(dt * dt / 6.0);
  sc.live = 1;
  return sc;
}

// accessors of the packed state
struct MxState {
  double* avg;   // [4][N]
  float* a32;    // [4][N]
  float* hi;     // [4][ML-1][N]
};
template <int ML>
__device__ __forceinline__ MxState mx_state(double* state, int N) {
  MxState st;
  st.avg = state;
  st.a32 = reinterpret_cast<float*>(state + 4 * (size_t)N);
  st.hi = st.a32 + 4 * (size_t)N;
  return st;
}
template <int ML>
__device__ __forceinline__ float& hi_at(const MxState& st, int N, int v, int l, int i) {
  return st.hi[((size_t)v * (ML - 1) + (l - 1)) * N + i];
}

// Zeroes the per-step diagnostics (and the status word when clear_status).
// Steps without diagnostics launch no reset: the moment kernel's last CTA
// zeroes each problem's speed maximum once it has read it, and the status word
// is sticky until the host reads it.
__global__ void k_reset_mx(DevWorkMx w, int nprob, int want_diag, int clear_status) {
  for (int p = threadIdx.x; p < nprob; p += blockDim.x) w.smax[p] = 0ull;
  if (threadIdx.x != 0) return;
  if (clear_status) *w.status = 0u;
  if (want_diag) {
    DiagBlock* d = reinterpret_cast<DiagBlock*>(w.diag);
    for (int c = 0; c < 4; ++c) d->sum[c] = 0.0;
    d->minr = d->minp = ~0ull;
    d->nmom = d->nedge = d->nsc = d->fb_mom = d->fb_edge = d->mlp_skip = 0ull;
  }
}

// CTA maximum of a non-negative value, one atomic per CTA (every thread of
// the CTA must call it; blockDim.x a multiple of 32, at most 1024)
__device__ __forceinline__ void block_max(float v, unsigned long long* dst) {
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) atomicMax(dst, (unsigned long long)__double_as_longlong((double)v * kSpeedInflate));
  }
  __syncthreads();   // red[] is reused by the next tile
}

// ---------------------------------------------------------- k_moment_mx
// Sec. 3.1.  FP32 screen, one thread per cell: a limiter point whose FP32
// density (pressure) clears its floor by more than the FP32 error bound
// cannot constrain theta -- the density is linear in theta, and the pressure
// along theta is concave (above the chord from the average's pressure,
// >= 2 eps_p, to the point's, > eps_p).  A cell all of whose points clear
// keeps theta = 1 exactly.  The other (cell, point) pairs are listed per
// warp in shared memory and evaluated in FP64, 32 pairs at a time, one per
// lane: Step 1 (density) then Step 2 (pressure of the density-limited
// state).  Each cell's theta is the minimum of its pairs' candidates, taken
// with shared-memory atomicMin on the bit patterns of the (positive)
// doubles, which is exact in any order: the same theta as a serial loop over
// all points.
template <int KD, int E, int ML, int NQ, int MQ>
__device__ __forceinline__ float moment_screen(const DevMesh& m, double* __restrict__ state, const StepArgs& a,
                                               const int i, unsigned& mr, unsigned& mp) {
  constexpr int NPT = NQ + E * MQ;
  const TablesF& t = c_tabf[KD];
  const int N = m.N;
  MxState st = mx_state<ML>(state, N);
  const float g = a.gamma_f, g1 = g - 1.0f;
  float a32[4], c[4][ML];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    a32[v] = st.a32[(size_t)v * N + i];
#pragma unroll
    for (int l = 1; l < ML; ++l) c[v][l] = hi_at<ML>(st, N, v, l, i);
  }
  float smax = 0.0f;
  const float eps0 = a.eps0_f;
  const float ri = 1.0f / a32[0];
  const float kb = 0.5f * (a32[1] * a32[1] + a32[2] * a32[2]) * ri;
  const float pb = g1 * (a32[3] - kb);
  const bool avg_ok = a32[0] > 0.0f && pb > kTol * g1 * (fabsf(a32[3]) + kb);
  const float er = fminf(eps0, 0.5f * a32[0]) * (1.0f + kTol);
  const float ep = fminf(eps0, 0.5f * pb) * (1.0f + kTol);
  mr = 0u; mp = 0u;
  // S_v bounds |a_v| + sum_l |c_vl phi_l(p)| at every point, so the FP32
  // error of each point value is below 1e-5 S_v with a wide margin
  float S[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    float sa = fabsf(a32[v]);
#pragma unroll
    for (int l = 1; l < ML; ++l) sa = fmaf(fabsf(c[v][l]), c_phimax[KD][l], sa);
    S[v] = sa;
  }
#pragma unroll 1
  for (int p = 0; p < NPT; ++p) {
    float q[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float acc = a32[v];
#pragma unroll
      for (int l = 1; l < ML; ++l) acc = fmaf(c[v][l], t.phi[p][l], acc);
      q[v] = acc;
    }
    const float rinv = 1.0f / q[0];
    const float u = q[1] * rinv, vv = q[2] * rinv;
    const float k2 = q[1] * u + q[2] * vv;
    const float pp = g1 * (q[3] - 0.5f * k2);
    const float B = S[3] + fabsf(u) * S[1] + fabsf(vv) * S[2] + 0.5f * (u * u + vv * vv) * S[0];
    const bool rok = q[0] > er + kTol * S[0];
    const bool pok = rok && pp > ep + kTol * g1 * B;
    mr |= rok ? 0u : (1u << p);
    mp |= pok ? 0u : (1u << p);
    const float pc = pp > 0.0f ? pp : 0.0f;
    smax = fmaxf(smax, sqrtf(u * u + vv * vv) + sqrtf(g * pc * rinv));
  }
  if (!avg_ok) {                       // the averages themselves are too close to call in FP32
    mr = mp = NPT == 32 ? 0xffffffffu : ((1u << NPT) - 1u);
  }
  if (!(mr | mp)) smax = fmaxf(smax, speedf(g, a32[0], a32[1], a32[2], a32[3]));
  return smax;
}

// Runs f(cell_lane, point) once for every set bit of every lane's mask,
// spread over the warp's lanes (list: the warp's shared scratch, >= 32 * 32
// entries).  All 32 lanes must call it.
template <class F>
__device__ __forceinline__ void warp_pairs(unsigned mask, unsigned short* list, F&& f) {
  const int lane = threadIdx.x & 31;
  const int cnt = __popc(mask);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  int off = incl - cnt;
  while (mask) {
    const int p = __ffs(mask) - 1;
    mask &= mask - 1;
    list[off++] = (unsigned short)((lane << 8) | p);
  }
  __syncwarp();
  for (int k = lane; k < total; k += 32) {
    const unsigned e = list[k];
    f((int)(e >> 8), (int)(e & 255u));
  }
  __syncwarp();
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(unsigned long long u) { return __longlong_as_double((long long)u); }

template <int KD, int E, int ML, int NQ, int MQ>
__global__ void __launch_bounds__(128, 6) k_moment_mx(const DevMesh m, const DevWorkMx w, double* __restrict__ state,
                                                   const StepArgs a, double* __restrict__ theta_out) {
  constexpr int NPT = NQ + E * MQ;
  static_assert(NPT <= 32, "a cell's limiter points fit one 32-bit mask");
  __shared__ unsigned short pair_list[4][32 * 32];
  __shared__ unsigned long long th_slot[4][32];
  __shared__ double thr_s[4][32], pb_s[4][32];
  const TablesF& t = c_tabf[KD];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  DiagBlock* dg = reinterpret_cast<DiagBlock*>(w.diag);
  const int N = m.N;
  MxState st = mx_state<ML>(state, N);
  const double gd1 = a.gamma - 1.0;
  for (int tl = blockIdx.x; tl < m.ntiles; tl += gridDim.x) {
    const int4 tile = m.tiles[tl];
    // a problem whose timed run has ended: nothing to do (uniform over the CTA)
    if (a.timed && !(__ldcg(a.tclock + 4 * tile.z) < a.t_end)) continue;
    const int i = tile.x + threadIdx.x;
    const int wbase = tile.x + warp * 32;      // element of lane 0 of this warp
    float sm = 0.0f;
    unsigned mr = 0u, mp = 0u;
    if ((int)threadIdx.x < tile.y) sm = moment_screen<KD, E, ML, NQ, MQ>(m, state, a, i, mr, mp);
    bool need = (mr | mp) != 0u;
    if (__any_sync(0xffffffffu, need)) {
      // FP64 averages of the cells that need the FP64 path
      bool bad = false;
      if (need) {
        const double rb = st.avg[i], mb = st.avg[(size_t)N + i], nb = st.avg[2 * (size_t)N + i],
                     eb = st.avg[3 * (size_t)N + i];
        const double pb = rb > 0.0 ? gd1 * (eb - 0.5 * (mb * mb + nb * nb) / rb) : -1.0;
        bad = !(rb > 0.0) || !(pb > 0.0);
        if (bad) mr = mp = 0u;
        pb_s[warp][lane] = pb;
      }
      th_slot[warp][lane] = dbits(1.0);
      __syncwarp();
      // Step 1: density candidates
      warp_pairs(mr, pair_list[warp], [&](int cl, int p) {
        const int ci = wbase + cl;
        const double rb = st.avg[ci];
        double d = 0.0;
#pragma unroll
        for (int l = 1; l < ML; ++l) d = fma((double)hi_at<ML>(st, N, 0, l, ci), c_phid[KD][p][l], d);
        const double rm = rb + d;
        const double er = fmin(a.eps0, 0.5 * rb);
        if (rm < er) atomicMin(&th_slot[warp][cl], dbits((rb - er) / (rb - rm)));
      });
      const double thr = bitsd(th_slot[warp][lane]);
      thr_s[warp][lane] = thr;
      __syncwarp();
      // Step 2: pressure candidates of the density-limited state (th starts at thr)
      warp_pairs(mp, pair_list[warp], [&](int cl, int p) {
        const int ci = wbase + cl;
        const double thr_c = thr_s[warp][cl], pb = pb_s[warp][cl];
        double d[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          double acc = 0.0;
#pragma unroll
          for (int l = 1; l < ML; ++l) acc = fma((double)hi_at<ML>(st, N, v, l, ci), c_phid[KD][p][l], acc);
          d[v] = acc;
        }
        const double rb = st.avg[ci], mb = st.avg[(size_t)N + ci], nb = st.avg[2 * (size_t)N + ci],
                     eb = st.avg[3 * (size_t)N + ci];
        const double r = rb + thr_c * d[0], mm = mb + thr_c * d[1], nn = nb + thr_c * d[2], ee = eb + thr_c * d[3];
        const double pt = gd1 * (ee - 0.5 * (mm * mm + nn * nn) / r);
        const double ep = fmin(a.eps0, 0.5 * pb);
        if (pt < ep)
          atomicMin(&th_slot[warp][cl], dbits(a.moment_exact ? exact_root_theta(rb, mb, nb, eb, d, ep / gd1, thr_c)
                                                             : thr_c * (pb - ep) / (pb - pt)));
      });
      if (need) {
        double th = bad ? 0.0 : fmax(bitsd(th_slot[warp][lane]), 0.0);
        atomicAdd(&dg->fb_mom, 1ull);
        if (bad) atomicOr(w.status, (unsigned)LXW_ST_NONPOSITIVE);
        // speeds of the limited state (FP32)
        const float g = a.gamma_f, thf = (float)th;
        float a32[4], c[4][ML];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          a32[v] = st.a32[(size_t)v * N + i];
#pragma unroll
          for (int l = 1; l < ML; ++l) c[v][l] = hi_at<ML>(st, N, v, l, i);
        }
        sm = a32[0] > 0.0f ? speedf(g, a32[0], a32[1], a32[2], a32[3]) : 0.0f;
        unsigned floor_pts = 0u;
#pragma unroll 1
        for (int p = 0; p < NPT; ++p) {
          float q[4];
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            float acc = 0.0f;
#pragma unroll
            for (int l = 1; l < ML; ++l) acc += c[v][l] * t.phi[p][l];
            q[v] = a32[v] + thf * acc;
          }
          const float k2 = q[1] * q[1] + q[2] * q[2];
          const float p32 = (g - 1.0f) * (q[3] - 0.5f * k2 / q[0]);
          // resolved in FP32: rho well above the cancellation of its own sum, p
          // well above that of E - |M|^2/(2 rho) (both within ~1e-5 then)
          if (q[0] > 1e-2f * a32[0] && p32 > 1e-2f * q[3]) sm = fmaxf(sm, speedf(g, q[0], q[1], q[2], q[3]));
          else floor_pts |= 1u << p;
        }
        // limited points near vacuum or the pressure floor: their density or
        // pressure cancels below the FP32 rounding, so their speed comes from the
        // FP64 point state (FP64 averages, the unlimited modes from memory, the
        // FP64 basis)
#pragma unroll 1
        for (unsigned fm = floor_pts; fm; fm &= fm - 1u) {
          const int p = __ffs(fm) - 1;
          double r[4];
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            double acc = 0.0;
#pragma unroll
            for (int l = 1; l < ML; ++l) acc = fma((double)hi_at<ML>(st, N, v, l, i), c_phid[KD][p][l], acc);
            r[v] = st.avg[(size_t)v * N + i] + th * acc;
          }
          if (r[0] > 0.0) {
            const double m2 = r[1] * r[1] + r[2] * r[2];
            const double rp = fmax(gd1 * (r[0] * r[3] - 0.5 * m2), 0.0);   // rho p
            sm = fmaxf(sm, (float)((sqrt(m2) + sqrt(a.gamma * rp)) / r[0]));
          }
        }
        if (th < 1.0) {
#pragma unroll
          for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int l = 1; l < ML; ++l) hi_at<ML>(st, N, v, l, i) = (float)(th * (double)hi_at<ML>(st, N, v, l, i));
          if (a.want_diag) atomicAdd(&dg->nmom, 1ull);
        }
        if (theta_out) theta_out[i] = th;
      }
      __syncwarp();
    }
    if (!need && (int)threadIdx.x < tile.y && theta_out) theta_out[i] = 1.0;
    block_max(sm, &w.smax[tile.z]);
  }
  // The last CTA to finish (its maxima, like every other CTA's, are in before
  // its count) turns each problem's maximum into (s, dt) and clears it for the
  // next step.  No CTA waits on another.
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(w.done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    for (int p = threadIdx.x; p < m.nprob; p += blockDim.x) {
      w.scal[p] = make_scal(m, w, a, p);
      w.smax[p] = 0ull;
    }
    if (threadIdx.x == 0) *w.done = 0u;
  }
}

// ---------------------------------------------------------- k_ck_mx
// Sec. 2.2-2.3 in FP32.  div F^h is a polynomial of degree deg-1 and so lies
// in the modal space: q_t = -div F^h and q_tt = -div (F_t)^h are carried as
// modal coefficients Qt, Qtt, accumulated straight from the contravariant
// fluxes at the interior points with the weighted differentiation tables
// (the same values as projecting F and differentiating the expansion, with
// fewer operations and 24 live coefficients per field instead of 48).
// Then F_T at every point, the volume integral added to the FP32 higher
// modes, and traces (q, n_out.F_T) at the edge points.
// ORD4: fourth order in time, Qttt = modal coefficients of q_ttt = -div
// (F_tt)^h accumulated like Qt and Qtt, and dt^3/24 F_ttt added to F_T.
template <int KD, int E, int ML, int NQ, int MQ, bool ORD4 = false>
__device__ __forceinline__ void ck_elem(const DevMesh& m, const DevWorkMx& w, double* __restrict__ state,
                                        const StepArgs& a, const int i, const ScalMx& sc) {
  constexpr int NPT = NQ + E * MQ;
  const TablesF& t = c_tabf[KD];
  const int N = m.N;
  MxState st = mx_state<ML>(state, N);
  const float g1 = a.gamma_f - 1.0f;
  const float dt = sc.dt32, c1 = sc.c1, c2 = sc.c2;
  float c[4][ML];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    c[v][0] = st.a32[(size_t)v * N + i];
#pragma unroll
    for (int l = 1; l < ML; ++l) c[v][l] = hi_at<ML>(st, N, v, l, i);
  }
  const float jxx = m.jinv32[i], jxy = m.jinv32[N + i];
  const float jyx = m.jinv32[2 * N + i], jyy = m.jinv32[3 * N + i];
  // pass 1: Qt = modal coefficients of q_t = -div F^h
  float Qt[4][ML];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) Qt[v][l] = 0.0f;
#pragma unroll 1
  for (int k = 0; k < NQ; ++k) {
    float q[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float acc = 0.0f;
#pragma unroll
      for (int l = 0; l < ML; ++l) acc = fmaf(c[v][l], t.phi[k][l], acc);
      q[v] = acc;
    }
    PtF s = ptf(g1, q[0], q[1], q[2], q[3]);
    float F[4], G[4];
    fluxf(s, F, G);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float fx = jxx * F[v] + jxy * G[v], fy = jyx * F[v] + jyy * G[v];
#pragma unroll
      for (int l = 0; l < ML; ++l) Qt[v][l] = fmaf(-fx, c_wd[KD][0][k][l], fmaf(-fy, c_wd[KD][1][k][l], Qt[v][l]));
    }
  }
  // pass 2: Qtt = modal coefficients of q_tt = -div (F'(q) q_t)^h
  float Qtt[4][ML];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) Qtt[v][l] = 0.0f;
#pragma unroll 1
  for (int k = 0; k < NQ; ++k) {
    float q[4], qt[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float acc = 0.0f, d1 = 0.0f;
#pragma unroll
      for (int l = 0; l < ML; ++l) {
        acc = fmaf(c[v][l], t.phi[k][l], acc);
        d1 = fmaf(Qt[v][l], t.phi[k][l], d1);
      }
      q[v] = acc; qt[v] = d1;
    }
    PtF s = ptf(g1, q[0], q[1], q[2], q[3]);
    float F1[4], G1[4], du, dvv, dp;
    d1f(g1, s, qt, F1, G1, du, dvv, dp);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float fx = jxx * F1[v] + jxy * G1[v], fy = jyx * F1[v] + jyy * G1[v];
#pragma unroll
      for (int l = 0; l < ML; ++l) Qtt[v][l] = fmaf(-fx, c_wd[KD][0][k][l], fmaf(-fy, c_wd[KD][1][k][l], Qtt[v][l]));
    }
  }
  // pass 2b (ORD4): Qttt = modal coefficients of q_ttt = -div (F_tt)^h
  constexpr int M4 = ORD4 ? ML : 1;
  float Qttt[4][M4];
  if (ORD4) {
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int l = 0; l < M4; ++l) Qttt[v][l] = 0.0f;
#pragma unroll 1
    for (int k = 0; k < NQ; ++k) {
      float q[4], qt[4], qtt[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        float acc = 0.0f, e1 = 0.0f, e2 = 0.0f;
#pragma unroll
        for (int l = 0; l < ML; ++l) {
          const float ph = t.phi[k][l];
          acc = fmaf(c[v][l], ph, acc);
          e1 = fmaf(Qt[v][l], ph, e1);
          e2 = fmaf(Qtt[v][l], ph, e2);
        }
        q[v] = acc; qt[v] = e1; qtt[v] = e2;
      }
      PtF s = ptf(g1, q[0], q[1], q[2], q[3]);
      float F1[4], G1[4], F2[4], G2[4], F3[4], G3[4], du, dvv, dp, eu, ev, ep;
      d1f(g1, s, qt, F1, G1, du, dvv, dp);
      d2f(g1, s, qt, du, dvv, dp, F2, G2);
      d1f(g1, s, qtt, F3, G3, eu, ev, ep);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float Ftt = F2[v] + F3[v], Gtt = G2[v] + G3[v];
        const float fx = jxx * Ftt + jxy * Gtt, fy = jyx * Ftt + jyy * Gtt;
#pragma unroll
        for (int l = 0; l < M4; ++l) Qttt[v][l] = fmaf(-fx, c_wd[KD][0][k][l], fmaf(-fy, c_wd[KD][1][k][l], Qttt[v][l]));
      }
    }
  }
  const float c3 = dt * dt * dt * (1.0f / 24.0f);
  // pass 3: F_T at every point; volume integral (interior), traces (edges)
  float Vv[4][ML];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) Vv[v][l] = 0.0f;
#pragma unroll 1
  for (int p = 0; p < NPT; ++p) {
    float q[4], qt[4], qtt[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float acc = 0.0f, e1 = 0.0f, e2 = 0.0f;
#pragma unroll
      for (int l = 0; l < ML; ++l) {
        const float ph = t.phi[p][l];
        acc = fmaf(c[v][l], ph, acc);
        e1 = fmaf(Qt[v][l], ph, e1);
        e2 = fmaf(Qtt[v][l], ph, e2);
      }
      q[v] = acc; qt[v] = e1; qtt[v] = e2;
    }
    PtF s = ptf(g1, q[0], q[1], q[2], q[3]);
    float F[4], G[4], F1[4], G1[4], F2[4], G2[4], F3[4], G3[4];
    float du, dvv, dp, eu, ev, ep;
    fluxf(s, F, G);
    d1f(g1, s, qt, F1, G1, du, dvv, dp);
    d2f(g1, s, qt, du, dvv, dp, F2, G2);
    d1f(g1, s, qtt, F3, G3, eu, ev, ep);
    float FT[4], GT[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      FT[v] = F[v] + c1 * F1[v] + c2 * (F2[v] + F3[v]);
      GT[v] = G[v] + c1 * G1[v] + c2 * (G2[v] + G3[v]);
    }
    if (ORD4) {
      float qttt[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        float acc = 0.0f;
#pragma unroll
        for (int l = 0; l < M4; ++l) acc = fmaf(Qttt[v][l], t.phi[p][l], acc);
        qttt[v] = acc;
      }
      float A[4], B[4], Cm[4], Dm[4], Fq[4], Gq[4], fu, fv, fp;
      d3f(g1, s, qt, A, B);
      d11f(g1, s, qt, qtt, Cm, Dm);
      d1f(g1, s, qttt, Fq, Gq, fu, fv, fp);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        FT[v] += c3 * (A[v] + 3.0f * Cm[v] + Fq[v]);
        GT[v] += c3 * (B[v] + 3.0f * Dm[v] + Gq[v]);
      }
    }
    if (p < NQ) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        float fx = t.w[p] * (jxx * FT[v] + jxy * GT[v]);
        float fy = t.w[p] * (jyx * FT[v] + jyy * GT[v]);
#pragma unroll
        for (int l = 1; l < ML; ++l) Vv[v][l] = fmaf(fx, t.dxi[p][l], fmaf(fy, t.deta[p][l], Vv[v][l]));
      }
    } else {
      const int k = (p - NQ) / MQ, pe = (p - NQ) % MQ;
      const float nx = m.nrm32[(2 * k) * N + i], ny = m.nrm32[(2 * k + 1) * N + i];
      float* tr = w.trace + ((size_t)(k * MQ + pe) * 8) * N + i;
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
    for (int l = 1; l < ML; ++l) hi_at<ML>(st, N, v, l, i) = c[v][l] + dt * Vv[v][l];
}

template <int KD, int E, int ML, int NQ, int MQ, bool ORD4 = false>
__global__ void __launch_bounds__(128, ML == 6 ? 4 : 2) k_ck_mx(const DevMesh m, const DevWorkMx w,
                                                                double* __restrict__ state, const StepArgs a) {
  for (int tl = blockIdx.x; tl < m.ntiles; tl += gridDim.x) {
    const int4 tile = m.tiles[tl];
    if ((int)threadIdx.x < tile.y && w.scal[tile.z].live)
      ck_elem<KD, E, ML, NQ, MQ, ORD4>(m, w, state, a, tile.x + threadIdx.x, w.scal[tile.z]);
  }
}

// ---------------------------------------------------------- k_edge_mx
// Sec. 3.3 Step 3 in FP32 (LLF at the edge points in the owner's order, so
// the two sides produce exact negatives; f^LxW; edge integral of the higher
// modes) and Steps 4-5: an FP32 screen shows Lambda = 1 and mu_c = 1 for
// every corner with an error margin, else the FP64 algorithm runs.
template <int KD, int E, int ML, int NQ, int MQ>
__device__ __forceinline__ void edge_elem(const DevMesh& m, const DevWorkMx& w, double* __restrict__ state,
                                          const StepArgs& a, const int i, const int pid) {
  const TablesF& t = c_tabf[KD];
  const int N = m.N;
  MxState st = mx_state<ML>(state, N);
  const ScalMx sc = w.scal[pid];
  const float s = sc.s32, g1f = a.gamma_f - 1.0f;
  const float dta = sc.dt32 * m.inva32[i];
  float qb[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) qb[v] = st.a32[(size_t)v * N + i];
  // gather the neighbour indices and every trace value first (memory-level parallelism)
  int nb[E], nk[E];
#pragma unroll
  for (int k = 0; k < E; ++k) { nb[k] = m.nbr[k * N + i]; nk[k] = m.nbk[k * N + i]; }
  float Ei[4][ML];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) Ei[v][l] = 0.0f;
  float fW[E][4], fF[E][4];
  PtF sb = ptf(g1f, qb[0], qb[1], qb[2], qb[3]);
  float Fb[4], Gb[4];
  fluxf(sb, Fb, Gb);
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int j = nb[k], kj = nk[k];
    const float nx = m.nrm32[(2 * k) * N + i], ny = m.nrm32[(2 * k + 1) * N + i];
    const float ln = sqrtf(nx * nx + ny * ny);
    const float hs = 0.5f * s * ln;
    const bool owner = j < 0 || i < j || (i == j && k < kj);
    // slot qo holds edge point number qo in the owner's order (own point p)
    float qi[MQ][4], Fi[MQ][4], qx[MQ][4], Fx[MQ][4];
#pragma unroll
    for (int qo = 0; qo < MQ; ++qo) {
      const int pp = owner ? qo : MQ - 1 - qo;
      const float* tr = w.trace + ((size_t)(k * MQ + pp) * 8) * N + i;
#pragma unroll
      for (int v = 0; v < 4; ++v) { qi[qo][v] = tr[(size_t)v * N]; Fi[qo][v] = tr[(size_t)(4 + v) * N]; }
    }
    float qn[4];
    if (j >= 0) {
#pragma unroll
      for (int v = 0; v < 4; ++v) qn[v] = st.a32[(size_t)v * N + j];
#pragma unroll
      for (int qo = 0; qo < MQ; ++qo) {
        const int pp = owner ? qo : MQ - 1 - qo;
        const float* tj = w.trace + ((size_t)(kj * MQ + (MQ - 1 - pp)) * 8) * N + j;
#pragma unroll
        for (int v = 0; v < 4; ++v) { qx[qo][v] = tj[(size_t)v * N]; Fx[qo][v] = -tj[(size_t)(4 + v) * N]; }
      }
    } else {
      const float nxh = nx / ln, nyh = ny / ln;
      ghostq<float>(-1 - j, nxh, nyh, qb, qn, a.qin32);
#pragma unroll
      for (int pp = 0; pp < MQ; ++pp) {
        if (-1 - j == LXW_BC_REFLECT) {
          ghostq<float>(LXW_BC_REFLECT, nxh, nyh, qi[pp], qx[pp], a.qin32);
          float R[4];
          ghostq<float>(LXW_BC_REFLECT, nxh, nyh, Fi[pp], R, a.qin32);
#pragma unroll
          for (int v = 0; v < 4; ++v) Fx[pp][v] = -R[v];
        } else if (-1 - j == LXW_BC_INFLOW) {
          // the steady inflow state: q_t = q_tt = 0, so n.F_T = n.F(q_in)
#pragma unroll
          for (int v = 0; v < 4; ++v) { qx[pp][v] = a.qin32[v]; Fx[pp][v] = nx * a.fin32[v] + ny * a.gin32[v]; }
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v) { qx[pp][v] = qi[pp][v]; Fx[pp][v] = Fi[pp][v]; }
        }
      }
    }
    {  // FP32 Lax-Friedrichs flux, used only by the screen
      PtF sn = ptf(g1f, qn[0], qn[1], qn[2], qn[3]);
      float Fn[4], Gn[4];
      fluxf(sn, Fn, Gn);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        float ai = nx * Fb[v] + ny * Gb[v], an = nx * Fn[v] + ny * Gn[v];
        fF[k][v] = 0.5f * (ai + an) - hs * (qn[v] - qb[v]);
      }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) fW[k][v] = 0.0f;
#pragma unroll
    for (int qo = 0; qo < MQ; ++qo) {
      const int p = owner ? qo : MQ - 1 - qo;
      // dissipation speed: the local Lax-Friedrichs speed of the two traces,
      // at most the global s (or s itself under the literal reading)
      const float hp = a.llf_global ? hs : 0.5f * fminf(s, fmaxf(lf_speedf(a.gamma_f, qi[qo]), lf_speedf(a.gamma_f, qx[qo]))) * ln;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        float fs = __fmaf_rn(-hp, __fsub_rn(qx[qo][v], qi[qo][v]), __fmul_rn(0.5f, __fadd_rn(Fi[qo][v], Fx[qo][v])));
        fW[k][v] = __fmaf_rn(0.5f * t.ew[qo], fs, fW[k][v]);
        const float hw = 0.5f * t.ew[p] * fs;
#pragma unroll
        for (int l = 1; l < ML; ++l) Ei[v][l] = fmaf(hw, t.phi[NQ + k * MQ + p][l], Ei[v][l]);
      }
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int l = 1; l < ML; ++l) hi_at<ML>(st, N, v, l, i) -= dta * Ei[v][l];

  // ---- FP32 screen of Steps 4-5 (Lambda = 1 for all edges, mu = 1 for all corners)
  const float tol = kTol;
  const float Tdt = 1.0f / dta;
  float gam = Tdt * qb[0], negabs = 0.0f, errr = Tdt * fabsf(qb[0]);
  float Sv[4], ql[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) { Sv[v] = fabsf(qb[v]); ql[v] = qb[v]; }
#pragma unroll
  for (int k = 0; k < E; ++k) {
    gam -= fF[k][0];
    negabs += fmaxf(0.0f, fW[k][0] - fF[k][0]);
    errr += fabsf(fF[k][0]) + fabsf(fW[k][0]);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      ql[v] -= dta * fF[k][v];
      Sv[v] += dta * (fabsf(fF[k][v]) + fabsf(fW[k][v]));
    }
  }
  bool clear = gam - Tdt * a.eps0_f - negabs > 4.0f * tol * errr && ql[0] > tol * Sv[0];
  // kappa = min(eps0, p^LxF/2)/(gamma-1) of the FP64 solve, bounded from above
  const float kl = 0.5f * (ql[1] * ql[1] + ql[2] * ql[2]) / ql[0];
  const float pl32 = g1f * (ql[3] - kl);
  const float kap = fminf(a.eps0_f, 0.5f * pl32 + tol * g1f * (fabsf(ql[3]) + kl)) / g1f;
  const float herr = 2.0f * tol * (Sv[0] * Sv[3] + Sv[1] * Sv[1] + Sv[2] * Sv[2] + kap * Sv[0]);
  auto hval = [&](const float q[4]) { return q[0] * q[3] - 0.5f * (q[1] * q[1] + q[2] * q[2]) - kap * q[0]; };
  clear = clear && pl32 > 0.0f && hval(ql) > herr;
#pragma unroll
  for (int cm = 1; cm < (1 << E); ++cm) {
    float qc[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float acc = ql[v];
#pragma unroll
      for (int k = 0; k < E; ++k)
        if ((cm >> k) & 1) acc += dta * (fF[k][v] - fW[k][v]);
      qc[v] = acc;
    }
    clear = clear && qc[0] > tol * Sv[0] && hval(qc) > herr;
  }
  float prop[E];
  if (clear) {
#pragma unroll
    for (int k = 0; k < E; ++k) prop[k] = 1.0f;
  } else {
    // ---- FP64 path (Sec. 3.3 Steps 4-5 as in the FP64 form)
    atomicAdd(&reinterpret_cast<DiagBlock*>(w.diag)->fb_edge, 1ull);
    const double g1 = a.gamma - 1.0, s64 = sc.s, dt64 = sc.dt;
    const double area = m.area[i], dta64 = dt64 * m.inva[i];
    double qb64[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) qb64[v] = st.avg[(size_t)v * N + i];
    double fF64[E][4], fW64[E][4];
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int j = nb[k];
      const double nx = m.nrm[(2 * k) * N + i], ny = m.nrm[(2 * k + 1) * N + i];
      double qn[4];
      if (j >= 0) {
#pragma unroll
        for (int v = 0; v < 4; ++v) qn[v] = st.avg[(size_t)v * N + j];
      } else {
        const double ln = sqrt(nx * nx + ny * ny);
        ghostq<double>(-1 - j, nx / ln, ny / ln, qb64, qn, a.qin);
      }
      lxf64(g1, s64, nx, ny, qb64, qn, fF64[k]);
#pragma unroll
      for (int v = 0; v < 4; ++v) fW64[k][v] = (double)fW[k][v];
    }
    double Gam0 = area / dt64 * qb64[0];
#pragma unroll
    for (int k = 0; k < E; ++k) Gam0 -= fF64[k][0];
    if (Gam0 < 0.0) atomicOr(w.status, (unsigned)LXW_ST_CFL);
    double neg = 0.0;
#pragma unroll
    for (int k = 0; k < E; ++k) {
      double df = fF64[k][0] - fW64[k][0];
      if (df < 0.0) neg += df;
    }
    double ql64[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < E; ++k) acc += fF64[k][v];
      ql64[v] = qb64[v] - dta64 * acc;
    }
    double er = fmax(fmin(a.eps0, 0.5 * ql64[0]), 0.0);
    double lneg = 1.0;
    if (neg < 0.0) lneg = fmin(1.0, fmax(0.0, (Gam0 - area / dt64 * er) / (-neg)));
    double lam[E], dq[E][4];
#pragma unroll
    for (int k = 0; k < E; ++k) {
      lam[k] = (fF64[k][0] - fW64[k][0]) < 0.0 ? lneg : 1.0;
#pragma unroll
      for (int v = 0; v < 4; ++v) dq[k][v] = dta64 * lam[k] * (fF64[k][v] - fW64[k][v]);
    }
    const double pl = ql64[0] > 0.0 ? g1 * (ql64[3] - 0.5 * (ql64[1] * ql64[1] + ql64[2] * ql64[2]) / ql64[0]) : -1.0;
    double mmin[E];
#pragma unroll
    for (int k = 0; k < E; ++k) mmin[k] = 1.0;
    if (!(ql64[0] > 0.0) || !(pl > 0.0)) {
#pragma unroll
      for (int k = 0; k < E; ++k) mmin[k] = 0.0;
    } else {
      const double kap64 = fmin(a.eps0, 0.5 * pl) / g1;
      const double h0 = ql64[0] * ql64[3] - 0.5 * (ql64[1] * ql64[1] + ql64[2] * ql64[2]) - kap64 * ql64[0];
#pragma unroll 1
      for (int cm = 1; cm < (1 << E); ++cm) {
        double d[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 0; k < E; ++k)
          if ((cm >> k) & 1)
#pragma unroll
            for (int v = 0; v < 4; ++v) d[v] += dq[k][v];
        const double h1 = ql64[0] * d[3] + d[0] * ql64[3] - (ql64[1] * d[1] + ql64[2] * d[2]) - kap64 * d[0];
        const double h2 = d[0] * d[3] - 0.5 * (d[1] * d[1] + d[2] * d[2]);
        double mu = 1.0;
        if (!(ql64[0] + d[0] > 0.0) || h0 + h1 + h2 < 0.0) {
          double disc = fmax(h1 * h1 - 4.0 * h0 * h2, 0.0);
          double den = -h1 + sqrt(disc);
          mu = den > 0.0 ? fmin(1.0, fmax(0.0, 2.0 * h0 / den)) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < E; ++k)
          if ((cm >> k) & 1) mmin[k] = fmin(mmin[k], mu);
      }
    }
    // theta rounded down to FP32 keeps the update inside the positive box
#pragma unroll
    for (int k = 0; k < E; ++k) prop[k] = __double2float_rd(lam[k] * mmin[k]);
  }
#pragma unroll
  for (int k = 0; k < E; ++k) {
    w.prop[k * N + i] = prop[k];
#pragma unroll
    for (int v = 0; v < 4; ++v) w.fw[(size_t)(k * 4 + v) * N + i] = fW[k][v];
  }
}

// HI: the variant with more resident CTAs per SM (fewer registers, some
// spills), which pays on large meshes; the autotuner chooses
template <int KD, int E, int ML, int NQ, int MQ, bool HI>
__global__ void __launch_bounds__(128, ML == 6 ? (HI ? 5 : 4) : 3) k_edge_mx(const DevMesh m, const DevWorkMx w,
                                                                  double* __restrict__ state, const StepArgs a) {
  for (int tl = blockIdx.x; tl < m.ntiles; tl += gridDim.x) {
    const int4 tile = m.tiles[tl];
    if ((int)threadIdx.x < tile.y && w.scal[tile.z].live)
      edge_elem<KD, E, ML, NQ, MQ>(m, w, state, a, tile.x + threadIdx.x, tile.z);
  }
}

// ---------------------------------------------------------- k_update_mx
// Sec. 3.3 Step 6 in FP64: theta_e = min of both proposals; the LxF flux is
// evaluated (FP64, from the old averages) only on edges with theta_e < 1.
// New averages go to avg_new (and an FP32 copy); the old ones stay readable
// for the neighbours.
template <int E, int ML>
__device__ __forceinline__ void update_elem(const DevMesh& m, const DevWorkMx& w, double* __restrict__ state,
                                            const StepArgs& a, const int i, const int pid) {
  const int N = m.N;
  MxState st = mx_state<ML>(state, N);
  // every load that does not depend on another first (f^LxW, averages, own
  // proposals, neighbour ids), then the neighbours' proposals
  float fwv[E][4];
#pragma unroll
  for (int k = 0; k < E; ++k)
#pragma unroll
    for (int v = 0; v < 4; ++v) fwv[k][v] = w.fw[(size_t)(k * 4 + v) * N + i];
  double qb[4], acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int v = 0; v < 4; ++v) qb[v] = st.avg[(size_t)v * N + i];
  int nb[E], nk[E];
  float th[E];
#pragma unroll
  for (int k = 0; k < E; ++k) { nb[k] = m.nbr[k * N + i]; nk[k] = m.nbk[k * N + i]; th[k] = w.prop[k * N + i]; }
  bool all_one = true;
#pragma unroll
  for (int k = 0; k < E; ++k) {
    if (nb[k] >= 0) th[k] = fminf(th[k], w.prop[nk[k] * N + nb[k]]);
    all_one = all_one && th[k] == 1.0f;
    if (a.theta_edge) a.theta_edge[(size_t)i * E + k] = th[k];
  }
  if (all_one) {
    // the common case: f^LxW only.  The E FP32 values are summed without
    // rounding error (Knuth's TwoSum in FP32 gives sum = hi + lo exactly up
    // to the last addition of the small parts), so only hi and lo go through
    // the slow FP64 pipe; the cell's flux sum keeps its FP64 accuracy and
    // both sides of an edge still add exact negatives.
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float hi = fwv[0][v], lo = 0.0f;
#pragma unroll
      for (int k = 1; k < E; ++k) {
        const float b = fwv[k][v];
        const float s1 = __fadd_rn(hi, b);
        const float bb = __fsub_rn(s1, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s1, bb)), __fsub_rn(b, bb));
        hi = s1;
        lo = __fadd_rn(lo, err);
      }
      acc[v] = (double)hi + (double)lo;
    }
  } else {
    const ScalMx sc = w.scal[pid];
    const double g1 = a.gamma - 1.0;
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int j = nb[k];
      double fw[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) fw[v] = (double)fwv[k][v];
      if (th[k] < 1.0f) {
        if (a.want_diag && (j < 0 || i < j || (i == j && k < nk[k])))
          atomicAdd(&reinterpret_cast<DiagBlock*>(w.diag)->nedge, 1ull);
        const double nx = m.nrm[(2 * k) * N + i], ny = m.nrm[(2 * k + 1) * N + i];
        double qn[4], ff[4];
        if (j >= 0) {
#pragma unroll
          for (int v = 0; v < 4; ++v) qn[v] = st.avg[(size_t)v * N + j];
        } else {
          const double ln = sqrt(nx * nx + ny * ny);
          ghostq<double>(-1 - j, nx / ln, ny / ln, qb, qn, a.qin);
        }
        lxf64(g1, sc.s, nx, ny, qb, qn, ff);
        const double t = (double)th[k];
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] += t * fw[v] + (1.0 - t) * ff[v];
      } else {
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] += fw[v];
      }
    }
  }
  const double dta = w.scal[pid].dt * m.inva[i];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const double an = qb[v] - dta * acc[v];
    w.avg_new[(size_t)v * N + i] = an;
    w.avgn32[(size_t)v * N + i] = (float)an;
  }
}

// six resident CTAs per SM (80 registers): more warps hide the gathers' latency
// (update 86 -> 70 us on 1024^2 squares); small spills only in the theta < 1 path
template <int E, int ML>
__global__ void __launch_bounds__(128, 6) k_update_mx(const DevMesh m, const DevWorkMx w, double* __restrict__ state,
                                                   const StepArgs a) {
  // the gated shock limiter's list of this step starts empty (the shock
  // kernels run after this one)
  if (blockIdx.x == 0 && threadIdx.x == 0) *w.gate_count = 0u;
  for (int tl = blockIdx.x; tl < m.ntiles; tl += gridDim.x) {
    const int4 tile = m.tiles[tl];
    if ((int)threadIdx.x < tile.y && w.scal[tile.z].live) update_elem<E, ML>(m, w, state, a, tile.x + threadIdx.x, tile.z);
  }
}

// ---------------------------------------------------------- learned gate
// Features of a cell at the shock limiter's input (all clipped to [-8, 8]):
// rho and E higher modes over their averages (first 5 modes), the first two
// higher modes of the momenta over rho_avg*(|u_avg| + c_avg), neighbour
// averages of rho and E relative to the cell's (missing neighbours 0),
// alpha / rho_avg and the internal-energy fraction p_avg / ((gamma-1) E_avg).
template <int E, int ML>
__device__ __forceinline__ void cell_features(const float c[4][ML], const float nr[4], const float ne[4], float g,
                                              float al, float f[kMlpIn]) {
  const float r = c[0][0], e = c[3][0];
  const float ri = 1.0f / r, ei = 1.0f / e;
  const float u = c[1][0] * ri, v = c[2][0] * ri;
  const float p = fmaxf((g - 1.0f) * (e - 0.5f * r * (u * u + v * v)), 0.0f);
  const float U = sqrtf(u * u + v * v) + sqrtf(g * p * ri);
  const float mi = 1.0f / fmaxf(r * U, 1e-30f);
#pragma unroll
  for (int l = 1; l <= 5; ++l) {
    f[l - 1] = (l < ML) ? c[0][l] * ri : 0.0f;
    f[4 + l] = (l < ML) ? c[3][l] * ei : 0.0f;
  }
  f[10] = c[1][1] * mi; f[11] = c[2][1] * mi; f[12] = c[1][2] * mi; f[13] = c[2][2] * mi;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    f[14 + k] = (k < E && nr[k] > 0.0f) ? nr[k] * ri - 1.0f : 0.0f;
    f[18 + k] = (k < E && nr[k] > 0.0f) ? ne[k] * ei - 1.0f : 0.0f;
  }
  f[22] = al * ri;
  f[23] = p / ((g - 1.0f) * e);
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) f[k] = fminf(8.0f, fmaxf(-8.0f, f[k]));
}

// ---- tensor-core inference of the gate (tcgen05, BF16 operands, FP32 in TMEM)
// A CTA of 128 threads evaluates the network for 128 cells at a time, one
// cell per thread = one TMEM lane:
//   H1 = relu(X W1 + b1):  X [128 x 32] (24 features, zero padded) in shared
//        memory, W1^T [64 x 32]; D = 64 FP32 columns of TMEM
//   H2 = relu(H1 W2 + b2): H1 rounded to BF16 into shared memory [128 x 64],
//        W2^T [64 x 64]; D reuses the same 64 columns
//   theta_hat = sigmoid(H2 . w3 + b3) on the CUDA cores, read back with tcgen05.ld.
// One thread issues the MMAs and commits them to an mbarrier; every wait is
// bounded (kGateWaitCycles), after which the CTA stops, flags LXW_ST_TIMEOUT,
// waits once more for its own MMAs and copies and frees its TMEM.
constexpr int kGateRows = 128;
constexpr int kGateTmemCols = 64;
constexpr long long kGateWaitCycles = 2000000000ll;   // ~1 s at 2 GHz
struct GateTile {
  GateWeights w;                                        // filled by one bulk async copy
  alignas(128) unsigned short a1[kGateRows * kGateK1];  // features, core-matrix layout
  alignas(128) unsigned short a2[kGateRows * kMlpH];    // hidden layer 1, core-matrix layout
  alignas(8) unsigned long long wbar, mbar;
  unsigned tmem;
};
static_assert(sizeof(GateWeights) % 16 == 0, "bulk copies move multiples of 16 bytes");
// instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28
constexpr unsigned kGateIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(kMlpH >> 3) << 17) |
                                ((unsigned)(kGateRows >> 4) << 24);

__device__ __forceinline__ unsigned short f2bf(float x) {
  unsigned u = __float_as_uint(x);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (unsigned short)(u >> 16);
}
__device__ __forceinline__ unsigned pack2(unsigned short lo, unsigned short hi) { return (unsigned)lo | ((unsigned)hi << 16); }
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K) and stride (8-row)
// byte offsets, each >> 4; bits 46-48 = 0b001; no swizzle, base offset 0
__device__ __forceinline__ unsigned long long umma_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr >> 4) & 0x3fffu) | ((unsigned long long)((lbo >> 4) & 0x3fffu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void umma_bf16(unsigned tmem_d, unsigned long long ad, unsigned long long bd, unsigned acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(kGateIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(unsigned a, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned a, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(a), "r"(phase)
      : "memory");
  return ok != 0u;
}
// true once the phase completed, false after `limit` SM cycles
__device__ __forceinline__ bool mbar_wait(unsigned a, unsigned phase, long long limit = kGateWaitCycles) {
  const long long t0 = clock64();
  while (!mbar_try(a, phase))
    if (clock64() - t0 > limit) return false;
  return true;
}
// 16 consecutive FP32 columns of this thread's TMEM lane; the wait carries the
// registers so that no use can be scheduled before it
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float v[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])
               :
               : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// the gate's features of element i at the shock limiter's input (false: no features, run the limiter)
template <int E, int ML>
__device__ __forceinline__ bool gate_features(const DevMesh& m, const DevWorkMx& w, const double* __restrict__ state,
                                              const StepArgs& a, const int i, float f[kMlpIn]) {
  const int N = m.N;
  MxState st = mx_state<ML>(const_cast<double*>(state), N);
  float c[4][ML];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    c[v][0] = w.avgn32[(size_t)v * N + i];
#pragma unroll
    for (int l = 1; l < ML; ++l) c[v][l] = hi_at<ML>(st, N, v, l, i);
  }
  if (!(c[0][0] > 0.0f) || !(c[3][0] > 0.0f)) return false;
  float nr[4] = {0.0f, 0.0f, 0.0f, 0.0f}, ne[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const float an[4] = {c[0][0], c[1][0], c[2][0], c[3][0]};
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int j = m.nbr[k * N + i];
    float qn[4];
    if (j >= 0) {
#pragma unroll
      for (int v = 0; v < 4; ++v) qn[v] = w.avgn32[(size_t)v * N + j];
    } else {
      const float nx = m.nrm32[(2 * k) * N + i], ny = m.nrm32[(2 * k + 1) * N + i];
      const float ln = sqrtf(nx * nx + ny * ny);
      ghostq<float>(-1 - j, nx / ln, ny / ln, an, qn, a.qin32);
    }
    nr[k] = qn[0]; ne[k] = qn[3];
  }
  const float dx = m.sdx32[i];
  cell_features<E, ML>(c, nr, ne, a.gamma_f, a.alpha0_f * dx * sqrtf(dx), f);
  return true;
}

// Exact shortcut of the shock limiter (Sec. 4.1, reading G14).  Its bounds
// satisfy M >= w_avg + alpha and m <= w_avg - alpha, so theta_sc = 1 whenever
// every primitive moves by at most alpha over the cell's points.  Per-cell
// bounds of the conserved excursions D_v >= |sum_l c_vl phi_l(p)| give those
// of the primitives: u_p - u = (dm_x - u drho) / rho_p, and
// p_p - p = (g-1)(dE - u.dm + |u|^2 drho / 2) - (g-1)|dm - u drho|^2 / (2 rho_p).
// The margins (1e-5 of the magnitudes) cover the FP32 evaluation of the full
// path, which then returns exactly 1 as well.  c[v][0] holds the averages.
template <int KD, int ML>
__device__ __forceinline__ bool shock_screen(const float c[4][ML], const PtF& sb, float g1, float al) {
  float D[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    float d = 0.0f;
#pragma unroll
    for (int l = 1; l < ML; ++l) d = fmaf(fabsf(c[v][l]), c_phimax[KD][l], d);
    D[v] = d * (1.0f + kTol);
  }
  const float rmin = sb.r - D[0] - kTol * sb.r;
  if (!(rmin > 0.0f && D[0] + kTol * (sb.r + D[0] + al) <= al)) return false;
  const float au = fabsf(sb.u), av = fabsf(sb.v);
  const float bu = D[1] + au * D[0], bv = D[2] + av * D[0];
  const float eu = bu / rmin, ev = bv / rmin;
  const float ep = g1 * (D[3] + au * D[1] + av * D[2] + 0.5f * (au * au + av * av) * D[0]) +
                   g1 * (bu * bu + bv * bv) / (2.0f * rmin);
  const float mp = g1 * (fabsf(c[3][0]) + D[3] + (fabsf(c[1][0]) + D[1]) * (au + eu) +
                         (fabsf(c[2][0]) + D[2]) * (av + ev));
  return eu + kTol * (au + eu + al) <= al && ev + kTol * (av + ev + al) <= al &&
         ep + kTol * (mp + fabsf(sb.p) + al) <= al;
}

// the screen for element i from the state (new averages, modes), or false
template <int KD, int ML>
__device__ __forceinline__ bool shock_screen_at(const DevMesh& m, const DevWorkMx& w, const double* __restrict__ state,
                                                const StepArgs& a, const int i) {
  const int N = m.N;
  MxState st = mx_state<ML>(const_cast<double*>(state), N);
  float c[4][ML];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    c[v][0] = w.avgn32[(size_t)v * N + i];
#pragma unroll
    for (int l = 1; l < ML; ++l) c[v][l] = hi_at<ML>(st, N, v, l, i);
  }
  if (!(c[0][0] > 0.0f)) return false;
  const float g1 = a.gamma_f - 1.0f;
  const PtF sb = ptf(g1, c[0][0], c[1][0], c[2][0], c[3][0]);
  const float dx = m.sdx32[i];
  return shock_screen<KD, ML>(c, sb, g1, a.alpha0_f * dx * sqrtf(dx));
}

template <int KD, int E, int ML, int NQ, int MQ>
__device__ __forceinline__ void shock_elem(const DevMesh& m, const DevWorkMx& w, double* __restrict__ state,
                                           const StepArgs& a, double* __restrict__ theta_out, const int limit,
                                           const int i, const bool skip, const bool defer = false) {
  constexpr int NPT = NQ + E * MQ;
  const TablesF& t = c_tabf[KD];
  const int N = m.N;
  MxState st = mx_state<ML>(state, N);
  // the new averages this cell commits at the end, loaded first (the stores
  // below may alias them as far as the compiler can tell)
  float an32[4];
  double an64[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) { an32[v] = w.avgn32[(size_t)v * N + i]; an64[v] = w.avg_new[(size_t)v * N + i]; }
  if (limit && skip) {
    if (theta_out) theta_out[i] = 1.0;
  } else if (limit) {
    const float g1 = a.gamma_f - 1.0f;
    float c[4][ML];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      c[v][0] = an32[v];
#pragma unroll
      for (int l = 1; l < ML; ++l) c[v][l] = hi_at<ML>(st, N, v, l, i);
    }
    float th = 1.0f;
    if (!(c[0][0] > 0.0f)) {
      th = 0.0f;
    } else {
      PtF sb = ptf(g1, c[0][0], c[1][0], c[2][0], c[3][0]);
      const float wb[4] = {sb.r, sb.u, sb.v, sb.p};
      const float dx = m.sdx32[i];
      const float al = a.alpha0_f * dx * sqrtf(dx);
      const bool clear = shock_screen<KD, ML>(c, sb, g1, al);
      if (!clear && defer) {
        // left to the gated limiter, which limits (or skips) and commits it
        w.gate_list[atomicAdd(w.gate_count, 1u)] = i;
        return;
      }
      float Mx[4], Mn[4], nr[4] = {0.0f, 0.0f, 0.0f, 0.0f}, ne[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int v = 0; v < 4; ++v) { Mx[v] = wb[v] + al; Mn[v] = wb[v] - al; }
      if (!clear) {
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const int j = m.nbr[k * N + i];
        float qn[4];
        if (j >= 0) {
#pragma unroll
          for (int v = 0; v < 4; ++v) qn[v] = w.avgn32[(size_t)v * N + j];
        } else {
          const float nx = m.nrm32[(2 * k) * N + i], ny = m.nrm32[(2 * k + 1) * N + i];
          const float ln = sqrtf(nx * nx + ny * ny);
          ghostq<float>(-1 - j, nx / ln, ny / ln, an32, qn, a.qin32);
        }
        nr[k] = qn[0]; ne[k] = qn[3];
        if (!(qn[0] > 0.0f)) continue;
        PtF sn = ptf(g1, qn[0], qn[1], qn[2], qn[3]);
        const float wn[4] = {sn.r, sn.u, sn.v, sn.p};
#pragma unroll
        for (int v = 0; v < 4; ++v) { Mx[v] = fmaxf(Mx[v], wn[v]); Mn[v] = fminf(Mn[v], wn[v]); }
      }
      {
        float hx[4], hn[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) { hx[v] = -3e38f; hn[v] = 3e38f; }
        bool bad = false;
#pragma unroll 1
        for (int p = 0; p < NPT; ++p) {
          float q[4];
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l < ML; ++l) acc = fmaf(c[v][l], t.phi[p][l], acc);
            q[v] = acc;
          }
          if (!(q[0] > 0.0f)) { bad = true; break; }
          PtF sp = ptf(g1, q[0], q[1], q[2], q[3]);
          const float wp[4] = {sp.r, sp.u, sp.v, sp.p};
#pragma unroll
          for (int v = 0; v < 4; ++v) { hx[v] = fmaxf(hx[v], wp[v]); hn[v] = fminf(hn[v], wp[v]); }
        }
        if (bad) {
          th = 0.0f;
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            if (hx[v] > wb[v]) th = fminf(th, (Mx[v] - wb[v]) / (hx[v] - wb[v]));
            if (hn[v] < wb[v]) th = fminf(th, (wb[v] - Mn[v]) / (wb[v] - hn[v]));
          }
          th = fmaxf(th, 0.0f);
        }
      }
      }   // !clear
    }
    if (th < 1.0f) {
#pragma unroll
      for (int v = 0; v < 4; ++v)
#pragma unroll
        for (int l = 1; l < ML; ++l) hi_at<ML>(st, N, v, l, i) = th * c[v][l];
      if (a.want_diag) atomicAdd(&reinterpret_cast<DiagBlock*>(w.diag)->nsc, 1ull);
    }
    if (theta_out) theta_out[i] = th;
  } else if (theta_out) {
    theta_out[i] = 1.0;
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    st.avg[(size_t)v * N + i] = an64[v];
    st.a32[(size_t)v * N + i] = an32[v];
  }
}

// The shock limiter behind the learned gate (features + network), over the
// mesh in tiles of 128 consecutive cells, persistent CTAs.  The exact screen
// (shock_screen) clears what it can; a tile holding any other cell computes
// its features and evaluates the network on the tensor cores; a cell the
// screen did not clear whose theta_hat >= 1 - tau (and whose averages are
// positive) keeps theta_sc = 1, every other cell runs the plain limiter;
// every cell commits its new averages.  On request it writes theta_hat and the
// features.  Without a network it writes the features (training pairs),
// runs the plain limiter everywhere and touches no tensor-core state.  If a
// device wait gives up, the CTA flags LXW_ST_TIMEOUT and runs the plain
// limiter on the rest of its cells.
// LIST: the cells come from w.gate_list (the ones the plain kernel's exact
// screen left, in any order), 128 per tile; a CTA with no tile leaves before
// it takes tensor memory or copies the weights.  Each row of a product
// depends only on its own cell, so the result is that of the full scan.
template <int KD, int E, int ML, int NQ, int MQ, bool HI, bool LIST = false>
__global__ void __launch_bounds__(kGateRows, HI ? 5 : 4) k_shock_gate_mx(const DevMesh m, const DevWorkMx w,
                                                             double* __restrict__ state, const StepArgs a,
                                                             double* __restrict__ theta_out) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const int N = m.N;
  if (a.timed && !w.scal[0].live) return;   // a timed run that has ended (one problem: the host checks)
  const int count = LIST ? (int)*w.gate_count : N;
  const int ntile = (count + kGateRows - 1) / kGateRows;
  if (LIST && (int)blockIdx.x >= ntile) return;
  if (a.gate_w == nullptr) {
    for (int i = blockIdx.x * blockDim.x + tid; i < N; i += gridDim.x * blockDim.x) {
      float f[kMlpIn];
      if (gate_features<E, ML>(m, w, state, a, i, f) && a.feat_out) {
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) a.feat_out[(size_t)i * kMlpIn + k] = f[k];
      }
      shock_elem<KD, E, ML, NQ, MQ>(m, w, state, a, theta_out, 1, i, false);
    }
    return;
  }
  extern __shared__ __align__(128) unsigned char gate_raw[];
  GateTile& g = *reinterpret_cast<GateTile*>(gate_raw);
  const unsigned wbar = smem_u32(&g.wbar), mbar = smem_u32(&g.mbar);
  if (tid == 0) {
    mbar_init(wbar, 1);
    mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // the weights travel while the first tiles are screened; the CTA waits
    // for them only at its first tile that needs the network
    constexpr unsigned bytes = (unsigned)sizeof(GateWeights);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(wbar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(&g.w)),
                 "l"(a.gate_w), "r"(bytes), "r"(wbar)
                 : "memory");
  }
  // tensor memory up front: taking it inside the tile loop, only where a
  // tile needs the network, measured slower (about 7 us per launch)
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&g.tmem)),
                 "r"(kGateTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = g.tmem;
  bool abort = false;
  bool wready = false;                    // the weight copy was seen complete
  bool mpending = false;                  // an MMA group committed but not seen complete
  unsigned phase = 0;
  const unsigned a1 = smem_u32(g.a1), a2 = smem_u32(g.a2), w1 = smem_u32(g.w.w1), w2 = smem_u32(g.w.w2);
  const unsigned lane_off = (unsigned)(warp * 32) << 16;
  unsigned long long skipped = 0;
  for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
    const int r = t * kGateRows + tid;
    const int i = LIST ? (r < count ? w.gate_list[r] : N) : r;
    // the network rules only on tiles holding a cell the exact screen cannot
    // clear (a listed cell is one)
    const bool clr = !LIST && i < N && shock_screen_at<KD, ML>(m, w, state, a, i);
    const bool inspect = a.gate_out || a.feat_out;          // every cell's theta_hat / features
    bool need_net = inspect || __syncthreads_or(i < N && !clr) != 0;
    if (need_net && !abort && !wready) {
      // test aid: a short wait on the MMA barrier before anything was
      // committed to it (nothing can arrive), so the timeout path runs
      if (a.gate_wait_test > 0) abort = __syncthreads_or(!mbar_wait(mbar, 0, a.gate_wait_test)) != 0;
      if (!abort) abort = __syncthreads_or(!mbar_wait(wbar, 0)) != 0;
      wready = !abort;
    }
    float f[kMlpIn];
    // features only where the answer is used (a cleared cell's row of the
    // product stays zero), or everywhere when inspected
    const bool ok = need_net && i < N && (!clr || inspect) && gate_features<E, ML>(m, w, state, a, i, f);
    if (ok && a.feat_out) {
#pragma unroll
      for (int k = 0; k < kMlpIn; ++k) a.feat_out[(size_t)i * kMlpIn + k] = f[k];
    }
    // the network is trusted only inside the envelope of its training features
    bool inside = ok && !abort;
    if (inside) {
#pragma unroll
      for (int k = 0; k < kMlpIn; ++k) inside = inside && f[k] >= g.w.lo[k] && f[k] <= g.w.hi[k];
    }
    if (!inspect && need_net) need_net = __syncthreads_or(inside && !clr) != 0;
    bool sk = false;
    if (need_net && !abort) {
      // this cell's features, BF16, as row tid of X (4 core matrices along K)
#pragma unroll
      for (int kb = 0; kb < kGateK1 / 8; ++kb) {
        uint4 q = make_uint4(0u, 0u, 0u, 0u);
        if (ok && kb * 8 < kMlpIn) {
          q.x = pack2(f2bf(f[kb * 8 + 0]), f2bf(f[kb * 8 + 1]));
          q.y = pack2(f2bf(f[kb * 8 + 2]), f2bf(f[kb * 8 + 3]));
          q.z = pack2(f2bf(f[kb * 8 + 4]), f2bf(f[kb * 8 + 5]));
          q.w = pack2(f2bf(f[kb * 8 + 6]), f2bf(f[kb * 8 + 7]));
        }
        *reinterpret_cast<uint4*>(&g.a1[umma_kmajor(tid, kb * 8, kGateK1)]) = q;
      }
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int s = 0; s < kGateK1 / 16; ++s)
          umma_bf16(tmem, umma_desc(a1 + 256u * s, 128u, 128u * (kGateK1 / 8)),
                    umma_desc(w1 + 256u * s, 128u, 128u * (kGateK1 / 8)), s > 0);
        umma_commit(mbar);
      }
      mpending = true;
      abort = __syncthreads_or(!mbar_wait(mbar, phase)) != 0;
    }
    if (need_net && !abort) {
      mpending = false;
      phase ^= 1u;
      tc_fence_after();
      // H1 row: bias, ReLU, BF16, 8 core matrices along K of the second product
#pragma unroll
      for (int c = 0; c < kMlpH / 16; ++c) {
        float v[16];
        tmem_ld16(tmem + lane_off + 16u * c, v);
        unsigned h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          h[j] = pack2(f2bf(fmaxf(v[2 * j] + g.w.b1[16 * c + 2 * j], 0.0f)),
                       f2bf(fmaxf(v[2 * j + 1] + g.w.b1[16 * c + 2 * j + 1], 0.0f)));
        *reinterpret_cast<uint4*>(&g.a2[umma_kmajor(tid, 16 * c, kMlpH)]) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(&g.a2[umma_kmajor(tid, 16 * c + 8, kMlpH)]) = make_uint4(h[4], h[5], h[6], h[7]);
      }
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int s = 0; s < kMlpH / 16; ++s)
          umma_bf16(tmem, umma_desc(a2 + 256u * s, 128u, 128u * (kMlpH / 8)),
                    umma_desc(w2 + 256u * s, 128u, 128u * (kMlpH / 8)), s > 0);
        umma_commit(mbar);
      }
      mpending = true;
      abort = __syncthreads_or(!mbar_wait(mbar, phase)) != 0;
    }
    if (need_net && !abort) {
      mpending = false;
      phase ^= 1u;
      tc_fence_after();
      float z = g.w.b3;
#pragma unroll
      for (int c = 0; c < kMlpH / 16; ++c) {
        float v[16];
        tmem_ld16(tmem + lane_off + 16u * c, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) z = fmaf(fmaxf(v[j] + g.w.b2[16 * c + j], 0.0f), g.w.w3[16 * c + j], z);
      }
      tc_fence_before();                   // these TMEM reads precede the next tile's MMAs
      const float th_hat = 1.0f / (1.0f + __expf(-z));
      sk = inside && !clr && th_hat >= 1.0f - a.mlp_tau;
      if (ok && a.gate_out) a.gate_out[i] = th_hat;
    }
    skipped += __popc(__ballot_sync(0xffffffffu, sk));
    // a cell the screen cleared keeps theta = 1 exactly as the limiter would
    if (i < N) shock_elem<KD, E, ML, NQ, MQ>(m, w, state, a, theta_out, 1, i, sk || clr);
  }
  if (tid == 0) {
    // the weight copy lands before the CTA leaves (its shared memory is
    // released at exit); after a timeout, give the copy / MMAs in flight one
    // more bounded wait and flag it
    if (!wready && !mbar_wait(wbar, 0)) abort = true;
    if (abort) {
      atomicOr(w.status, (unsigned)LXW_ST_TIMEOUT);
      if (mpending) mbar_wait(mbar, phase);
    }
  }
  if (a.want_diag && (tid & 31) == 0 && skipped)
    atomicAdd(&reinterpret_cast<DiagBlock*>(w.diag)->mlp_skip, skipped);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGateTmemCols) : "memory");
  }
}

// defer: cells the exact screen cannot clear go to the gated limiter's list
// (k_shock_gate_mx<..., LIST>) instead of being limited and committed here
template <int KD, int E, int ML, int NQ, int MQ>
__global__ void __launch_bounds__(128) k_shock_mx(const DevMesh m, const DevWorkMx w, double* __restrict__ state,
                                                  const StepArgs a, double* __restrict__ theta_out, int limit,
                                                  int defer) {
  for (int tl = blockIdx.x; tl < m.ntiles; tl += gridDim.x) {
    const int4 tile = m.tiles[tl];
    if ((int)threadIdx.x < tile.y && w.scal[tile.z].live)
      shock_elem<KD, E, ML, NQ, MQ>(m, w, state, a, theta_out, limit, tile.x + threadIdx.x, false, defer != 0);
  }
}

template <int ML>
__global__ void __launch_bounds__(256) k_diag_mx(const DevMesh m, const DevWorkMx w, const double* __restrict__ state,
                                                 double gamma) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = m.N;
  DiagBlock* d = reinterpret_cast<DiagBlock*>(w.diag);
  if (i < N) {
    double q[4];
    for (int v = 0; v < 4; ++v) q[v] = state[(size_t)v * N + i];
    double p = (gamma - 1.0) * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / q[0]);
    bool finite = true;
    for (int v = 0; v < 4; ++v) finite = finite && isfinite(q[v]);
    const float* hi = reinterpret_cast<const float*>(state + 4 * (size_t)N) + 4 * (size_t)N;
    for (int c = 0; c < 4 * (ML - 1); ++c) finite = finite && isfinite(hi[(size_t)c * N + i]);
    if (!finite) atomicOr(w.status, (unsigned)LXW_ST_NAN);
    const double ar = m.area[i];
    for (int v = 0; v < 4; ++v) atomicAdd(&d->sum[v], ar * q[v]);
    atomicMin(&d->minr, obits(q[0]));
    atomicMin(&d->minp, obits(p));
  }
}

// Q64[N][4][ML] (element-major, the ABI layout) <-> the mixed state layout,
// through shared memory so that both sides are read and written in
// consecutive words: 128 elements per CTA.  Q64 may be host memory mapped
// into the device's address space (pinned), read or written here directly.
constexpr int kPackRows = 128;
// vec: Q64 is 16-byte aligned (every CTA's block of 128 x 4 ML doubles then is)
template <int ML>
__global__ void __launch_bounds__(kPackRows) k_pack(int N, const double* __restrict__ Q64,
                                                    double* __restrict__ state, int vec) {
  __shared__ __align__(16) double buf[kPackRows * 4 * ML];
  const int base = blockIdx.x * kPackRows;
  const int n = min(kPackRows, N - base);
  const double* src = Q64 + (size_t)base * 4 * ML;
  if (vec) {
    const int pairs = n * 2 * ML;
    const double2* s2 = reinterpret_cast<const double2*>(src);
    double2* b2 = reinterpret_cast<double2*>(buf);
#pragma unroll 4
    for (int k = threadIdx.x; k < pairs; k += blockDim.x) b2[k] = s2[k];   // several loads in flight per thread
  } else {
#pragma unroll 4
    for (int k = threadIdx.x; k < n * 4 * ML; k += blockDim.x) buf[k] = src[k];
  }
  __syncthreads();
  if ((int)threadIdx.x < n) {
    const int i = base + threadIdx.x;
    float* a32 = reinterpret_cast<float*>(state + 4 * (size_t)N);
    float* hi = a32 + 4 * (size_t)N;
    const double* e = buf + threadIdx.x * 4 * ML;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double av = e[v * ML];
      state[(size_t)v * N + i] = av;
      a32[(size_t)v * N + i] = (float)av;
#pragma unroll
      for (int l = 1; l < ML; ++l) hi[((size_t)v * (ML - 1) + l - 1) * N + i] = (float)e[v * ML + l];
    }
  }
}

template <int ML>
__global__ void __launch_bounds__(kPackRows) k_unpack(int N, const double* __restrict__ state,
                                                      double* __restrict__ Q64, int vec) {
  __shared__ __align__(16) double buf[kPackRows * 4 * ML];
  const int base = blockIdx.x * kPackRows;
  const int n = min(kPackRows, N - base);
  if ((int)threadIdx.x < n) {
    const int i = base + threadIdx.x;
    const float* hi = reinterpret_cast<const float*>(state + 4 * (size_t)N) + 4 * (size_t)N;
    double* e = buf + threadIdx.x * 4 * ML;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      e[v * ML] = state[(size_t)v * N + i];
#pragma unroll
      for (int l = 1; l < ML; ++l) e[v * ML + l] = (double)hi[((size_t)v * (ML - 1) + l - 1) * N + i];
    }
  }
  __syncthreads();
  double* dst = Q64 + (size_t)base * 4 * ML;
  if (vec) {
    const int pairs = n * 2 * ML;
    double2* d2 = reinterpret_cast<double2*>(dst);
    const double2* b2 = reinterpret_cast<const double2*>(buf);
#pragma unroll 4
    for (int k = threadIdx.x; k < pairs; k += blockDim.x) d2[k] = b2[k];
  } else {
#pragma unroll 4
    for (int k = threadIdx.x; k < n * 4 * ML; k += blockDim.x) dst[k] = buf[k];
  }
}

inline int gridn(int N, int block) { return (N + block - 1) / block; }

template <int KD, int E, int ML, int NQ, int MQ>
int step_mx_impl(const DevMesh& m, const DevWorkMx& w, double* state, const StepArgs& a, cudaStream_t st, int block,
                 void** events, int upto) {
  const int grid = a.grid > 0 && a.grid < m.ntiles ? a.grid : m.ntiles;
  int ne = 0;
  auto mark = [&]() { if (events) cudaEventRecordWithFlags((cudaEvent_t)events[ne++], st, cudaEventRecordExternal); };
  auto ok = [&]() { return cudaGetLastError() == cudaSuccess ? 0 : -1; };
  mark();
  if (a.want_diag) k_reset_mx<<<1, 256, 0, st>>>(w, m.nprob, 1, 0);
  k_moment_mx<KD, E, ML, NQ, MQ><<<grid, block, 0, st>>>(m, w, state, a, a.theta_cell);
  mark();
  if (upto < 2) return ok();
  if (a.ck_order == 4)
    k_ck_mx<KD, E, ML, NQ, MQ, true><<<grid, block, 0, st>>>(m, w, state, a);
  else
    k_ck_mx<KD, E, ML, NQ, MQ><<<grid, block, 0, st>>>(m, w, state, a);
  mark();
  if (upto < 3) return ok();
  if (a.hi_occupancy)
    k_edge_mx<KD, E, ML, NQ, MQ, true><<<grid, block, 0, st>>>(m, w, state, a);
  else
    k_edge_mx<KD, E, ML, NQ, MQ, false><<<grid, block, 0, st>>>(m, w, state, a);
  mark();
  if (upto < 4) return ok();
  k_update_mx<E, ML><<<grid, block, 0, st>>>(m, w, state, a);
  mark();
  const int limit = a.shock_limiter && upto >= 5;
  double* tsc = a.theta_cell ? a.theta_cell + m.N : nullptr;
  if (limit && (a.gate_w || a.feat_out)) {
    // persistent CTAs, each copying the weights once and holding 64 TMEM
    // columns: a.gate_per_sm of them per SM (resident by occupancy, <= 8)
    const int ntile = (m.N + kGateRows - 1) / kGateRows;
    const int gg = std::max(1, std::min(ntile, std::max(a.gate_per_sm, 1) * std::max(a.sms, 1)));
    const size_t smem = a.gate_w ? sizeof(GateTile) : 0;
    if (a.gate_w && !a.gate_out && !a.feat_out && !a.gate_scan) {
      // the plain kernel screens every cell, commits the cleared ones and
      // lists the rest; the gate kernel takes only the listed cells
      k_shock_mx<KD, E, ML, NQ, MQ><<<grid, block, 0, st>>>(m, w, state, a, tsc, 1, 1);
      if (a.hi_occupancy)
        k_shock_gate_mx<KD, E, ML, NQ, MQ, true, true><<<gg, kGateRows, smem, st>>>(m, w, state, a, tsc);
      else
        k_shock_gate_mx<KD, E, ML, NQ, MQ, false, true><<<gg, kGateRows, smem, st>>>(m, w, state, a, tsc);
    } else if (a.hi_occupancy) {
      k_shock_gate_mx<KD, E, ML, NQ, MQ, true><<<gg, kGateRows, smem, st>>>(m, w, state, a, tsc);
    } else {
      k_shock_gate_mx<KD, E, ML, NQ, MQ, false><<<gg, kGateRows, smem, st>>>(m, w, state, a, tsc);
    }
  } else {
    k_shock_mx<KD, E, ML, NQ, MQ><<<grid, block, 0, st>>>(m, w, state, a, tsc, limit, 0);
  }
  mark();
  if (a.want_diag) k_diag_mx<ML><<<gridn(m.N, 256), 256, 0, st>>>(m, w, state, a.gamma);
  return ok();
}

template <int KD, int E, int ML, int NQ, int MQ>
int moment_mx_impl(const DevMesh& m, const DevWorkMx& w, double* state, const StepArgs& a, double* theta,
                   cudaStream_t st, int block) {
  const int grid = a.grid > 0 && a.grid < m.ntiles ? a.grid : m.ntiles;
  k_reset_mx<<<1, 256, 0, st>>>(w, m.nprob, 1, 1);
  k_moment_mx<KD, E, ML, NQ, MQ><<<grid, block, 0, st>>>(m, w, state, a, theta);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

#define LXW_DISPATCH_MX(kind, deg, CALL)                                \
  do {                                                                  \
    if (kind == LXW_KIND_QUAD && deg == 2) return CALL(0, 4, 6, 9, 3);   \
    if (kind == LXW_KIND_QUAD && deg == 3) return CALL(1, 4, 10, 16, 4); \
    if (kind == LXW_KIND_TRI && deg == 2) return CALL(2, 3, 6, 9, 3);    \
    if (kind == LXW_KIND_TRI && deg == 3) return CALL(3, 3, 10, 16, 4);  \
    return -2;                                                          \
  } while (0)

// Resident CTAs per SM of the gate kernel from its registers, shared memory
// and threads (the limits the hardware applies), capped by the 512 TMEM
// columns of an SM.  The shared-memory carveout is set to its maximum first.
template <int KD, int E, int ML, int NQ, int MQ, bool HI>
int gate_occupancy_impl() {
  auto fn = k_shock_gate_mx<KD, E, ML, NQ, MQ, HI>;
  auto fl = k_shock_gate_mx<KD, E, ML, NQ, MQ, HI, true>;   // the list form: same resources
  if (cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
          cudaSuccess ||
      cudaFuncSetAttribute(fl, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
          cudaSuccess)
    return -1;
  cudaFuncAttributes fa;
  int dev = 0, regs_sm = 0, smem_sm = 0, smem_rsv = 0, thr_sm = 0, blk_sm = 0;
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess)
    return -1;
  const int regs_cta = ((std::max(fa.numRegs, 1) * 32 + 255) / 256) * 256 * (kGateRows / 32);   // 256-register units per warp
  const int smem_cta = (int)sizeof(GateTile) + (int)fa.sharedSizeBytes + smem_rsv;
  int n = std::min({regs_sm / regs_cta, smem_sm / smem_cta, thr_sm / kGateRows, blk_sm});
  return std::min(n, 512 / kGateTmemCols);
}

int gate_occupancy(int kind, int deg, int hi) {
#define CALL_GOC(KD, E, ML, NQ, MQ) \
  (hi ? gate_occupancy_impl<KD, E, ML, NQ, MQ, true>() : gate_occupancy_impl<KD, E, ML, NQ, MQ, false>())
  LXW_DISPATCH_MX(kind, deg, CALL_GOC);
#undef CALL_GOC
}

int launch_step_mx(int kind, int deg, const DevMesh& m, const DevWorkMx& w, double* state, const StepArgs& a,
                   void* stream, int block, void** events, int upto) {
#define CALL_SMX(KD, E, ML, NQ, MQ) step_mx_impl<KD, E, ML, NQ, MQ>(m, w, state, a, (cudaStream_t)stream, block, events, upto)
  LXW_DISPATCH_MX(kind, deg, CALL_SMX);
#undef CALL_SMX
}

int launch_moment_limit_mx(int kind, int deg, const DevMesh& m, const DevWorkMx& w, double* state,
                           const StepArgs& a, double* theta, void* stream, int block) {
#define CALL_MMX(KD, E, ML, NQ, MQ) moment_mx_impl<KD, E, ML, NQ, MQ>(m, w, state, a, theta, (cudaStream_t)stream, block)
  LXW_DISPATCH_MX(kind, deg, CALL_MMX);
#undef CALL_MMX
}

int launch_pack(int ML, int N, const double* Q64, double* state, void* stream) {
  const int vec = (reinterpret_cast<uintptr_t>(Q64) & 15u) == 0;
  if (ML == 6)
    k_pack<6><<<gridn(N, kPackRows), kPackRows, 0, (cudaStream_t)stream>>>(N, Q64, state, vec);
  else
    k_pack<10><<<gridn(N, kPackRows), kPackRows, 0, (cudaStream_t)stream>>>(N, Q64, state, vec);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_unpack(int ML, int N, const double* state, double* Q64, void* stream) {
  const int vec = (reinterpret_cast<uintptr_t>(Q64) & 15u) == 0;
  if (ML == 6)
    k_unpack<6><<<gridn(N, kPackRows), kPackRows, 0, (cudaStream_t)stream>>>(N, state, Q64, vec);
  else
    k_unpack<10><<<gridn(N, kPackRows), kPackRows, 0, (cudaStream_t)stream>>>(N, state, Q64, vec);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int upload_tables_mx(int kind, int deg, const Tables& t) {
  const int kd = (kind == LXW_KIND_QUAD ? 0 : 2) + (deg == 3 ? 1 : 0);
  TablesF f{};
  for (int k = 0; k < kMaxQ; ++k) f.w[k] = (float)t.w[k];
  for (int k = 0; k < kMaxMQ; ++k) f.ew[k] = (float)t.ew[k];
  for (int p = 0; p < kMaxPts; ++p)
    for (int l = 0; l < kMaxML; ++l) {
      f.phi[p][l] = (float)t.phi[p][l];
      f.dxi[p][l] = (float)t.dxi[p][l];
      f.deta[p][l] = (float)t.deta[p][l];
    }
  if (cudaMemcpyToSymbol(c_tabf, &f, sizeof(TablesF), kd * sizeof(TablesF)) != cudaSuccess) return -1;
  DerivTables d;
  make_deriv_tables(t, d);
  float wd[2][kMaxQ][kMaxML];
  for (int c = 0; c < 2; ++c)
    for (int k = 0; k < kMaxQ; ++k)
      for (int l = 0; l < kMaxML; ++l) wd[c][k][l] = (float)d.W[c][k][l];
  if (cudaMemcpyToSymbol(c_wd, wd, sizeof(wd), kd * sizeof(wd)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_phid, t.phi, sizeof(double) * kMaxPts * kMaxML,
                         kd * sizeof(double) * kMaxPts * kMaxML) != cudaSuccess)
    return -1;
  float pm[kMaxML];
  for (int l = 0; l < kMaxML; ++l) {
    double mx = 0.0;
    for (int p = 0; p < kMaxPts; ++p) mx = std::max(mx, std::fabs(t.phi[p][l]));
    pm[l] = (float)(mx * (1.0 + 1e-6));   // rounded up
  }
  if (cudaMemcpyToSymbol(c_phimax, pm, sizeof(pm), kd * sizeof(pm)) != cudaSuccess) return -1;
  return 0;
}

}  // namespace lxw
