// lxw_flux3.cuh -- device helpers of the 3D forms (hexahedra and
// tetrahedra, FP64 and mixed): the Euler flux in three directions and along
// a normal, its first and second directional derivatives (the
// Cauchy-Kovalevskaya terms of Sec. 2.2), the wave speed and the local
// Lax-Friedrichs speed, the moment limiter of Sec. 3.1, and the FP32 screens
// of the mixed forms.  Included inside each kernel file's anonymous
// namespace.
#pragma once

__device__ __forceinline__ double speed_of3(double g, const double q[5]) {
  if (!(q[0] > 0.0)) return 0.0;
  const double ri = 1.0 / q[0];
  const double u = q[1] * ri, v = q[2] * ri, w = q[3] * ri;
  const double k2 = u * u + v * v + w * w;
  const double p = (g - 1.0) * (q[4] - 0.5 * q[0] * k2);
  return sqrt(k2) + (p > 0.0 ? sqrt(g * p * ri) : 0.0);
}

// fma / min / max in the argument's own precision (an unqualified fma on
// floats may resolve to the double function and run on the FP64 pipe).
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fminT(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float fminT(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double fmaxT(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float fmaxT(float a, float b) { return fmaxf(a, b); }

// A value the compiler must keep (in a register, or spilled) rather than
// recompute at each use: under register pressure it otherwise re-derives
// FP32 constants from FP64 sources (divisions, conversions) on the FP64 pipe.
__device__ __forceinline__ float opaque(float x) {
  asm volatile("" : "+f"(x));
  return x;
}
__device__ __forceinline__ double opaque(double x) {
  asm volatile("" : "+d"(x));
  return x;
}

// Explicitly rounded arithmetic in either precision: sign-symmetric, so
// operations on negated operands give exactly negated results.
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_sqrt(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float rn_sqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double rn_rcp(double a) { return __drcp_rn(a); }
__device__ __forceinline__ float rn_rcp(float a) { return __frcp_rn(a); }

// The local Lax-Friedrichs speed of a trace with explicitly rounded
// operations: both cells of a face evaluate it on the same two traces and
// must get the same value.
template <typename T>
__device__ __forceinline__ T lf_speed3(T g, const T q[5]) {
  if (!(q[0] > T(0))) return T(0);
  const T ri = rn_rcp(q[0]);
  const T u = rn_mul(q[1], ri), v = rn_mul(q[2], ri), w = rn_mul(q[3], ri);
  const T k2 = rn_add(rn_add(rn_mul(u, u), rn_mul(v, v)), rn_mul(w, w));
  const T p = rn_mul(g - T(1), rn_sub(q[4], rn_mul(T(0.5), rn_mul(q[0], k2))));
  const T c = p > T(0) ? rn_sqrt(rn_mul(rn_mul(g, p), ri)) : T(0);
  return rn_add(rn_sqrt(k2), c);
}

__device__ __forceinline__ void block_max3(double v, unsigned long long* dst) {
  // v >= 0: its bits order like the values
  __shared__ unsigned long long sm[32];
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t = __shfl_down_sync(0xffffffffu, b, o);
    b = t > b ? t : b;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sm[warp] = b;
  __syncthreads();
  if (warp == 0) {
    b = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long t = __shfl_down_sync(0xffffffffu, b, o);
      b = t > b ? t : b;
    }
    if (lane == 0) atomicMax(dst, b);
  }
}

// ---------------------------------------------------------------- flux
// Templated on the arithmetic type: double for the FP64 forms, float for the
// FP32 Cauchy-Kovalevskaya kernels of the mixed forms.
// Point state with its primitives.
template <typename T>
struct P3T {
  T q[5];
  T ri, u[3], p;
};
using P3 = P3T<double>;

template <typename T>
__device__ __forceinline__ P3T<T> make_p3(T g1, const T q[5]) {
  P3T<T> s;
#pragma unroll
  for (int v = 0; v < 5; ++v) s.q[v] = q[v];
  s.ri = T(1) / q[0];
#pragma unroll
  for (int d = 0; d < 3; ++d) s.u[d] = q[1 + d] * s.ri;
  s.p = g1 * (q[4] - T(0.5) * (q[1] * s.u[0] + q[2] * s.u[1] + q[3] * s.u[2]));
  return s;
}

// F_d(q), d = 0, 1, 2
template <typename T>
__device__ __forceinline__ void flux3(const P3T<T>& s, T F[3][5]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F[d][0] = s.q[1 + d];
#pragma unroll
    for (int e = 0; e < 3; ++e) F[d][1 + e] = s.q[1 + e] * s.u[d] + (e == d ? s.p : T(0));
    F[d][4] = (s.q[4] + s.p) * s.u[d];
  }
}

// F'(q) w; also the primitive increments du (velocity) and dp along w
template <typename T>
__device__ __forceinline__ void flux3_d1(T g1, const P3T<T>& s, const T w[5], T F[3][5], T du[3], T& dp) {
#pragma unroll
  for (int d = 0; d < 3; ++d) du[d] = (w[1 + d] - s.u[d] * w[0]) * s.ri;
  const T k2 = s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2];
  dp = g1 * (w[4] - (s.u[0] * w[1] + s.u[1] * w[2] + s.u[2] * w[3]) + T(0.5) * k2 * w[0]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F[d][0] = w[1 + d];
#pragma unroll
    for (int e = 0; e < 3; ++e) F[d][1 + e] = w[1 + e] * s.u[d] + s.q[1 + e] * du[d] + (e == d ? dp : T(0));
    F[d][4] = (w[4] + dp) * s.u[d] + (s.q[4] + s.p) * du[d];
  }
}

// F''(q)(w, w) from the increments of flux3_d1: along q + t w the density
// and momentum are linear, so u'' = -2 w_rho u' / rho and
// p'' = -(g-1)(m' . u' + m . u'' / 2)
template <typename T>
__device__ __forceinline__ void flux3_d2(T g1, const P3T<T>& s, const T w[5], const T du[3], T dp, T F[3][5]) {
  T d2u[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) d2u[d] = T(-2) * w[0] * du[d] * s.ri;
  const T d2p = -g1 * ((w[1] * du[0] + w[2] * du[1] + w[3] * du[2]) +
                       T(0.5) * (s.q[1] * d2u[0] + s.q[2] * d2u[1] + s.q[3] * d2u[2]));
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F[d][0] = T(0);
#pragma unroll
    for (int e = 0; e < 3; ++e) F[d][1 + e] = T(2) * w[1 + e] * du[d] + s.q[1 + e] * d2u[d] + (e == d ? d2p : T(0));
    F[d][4] = d2p * s.u[d] + T(2) * (w[4] + dp) * du[d] + (s.q[4] + s.p) * d2u[d];
  }
}

// ---------------------------------------------------------------- moment limiter
// Sec. 3.1 Steps 0-2 (Lemma 1's secant) on one cell's coefficients c[5][ML]
// (scaled in place when limited); load(p, ph) gives the basis values at
// limiter point p.  Returns theta (0 for a non-positive average, nonpos set)
// and smax = max |u| + c of the limited state over its average and points.
// One pass over the points yields the density minimum, the pressure
// proposal for an unlimited density and the wave speed, which is all a cell
// that is not limited needs; a limited cell takes the pressure pass with its
// density theta and a wave-speed pass over the scaled state.
template <int ML, int NPT, class Load>
__device__ __forceinline__ double moment_cell3(double c[5][ML], double g, double eps0, const Load& load, double& smax,
                                               bool& nonpos) {
  const double g1 = g - 1.0;
  const double pb = c[0][0] > 0.0
                        ? g1 * (c[4][0] - 0.5 * (c[1][0] * c[1][0] + c[2][0] * c[2][0] + c[3][0] * c[3][0]) / c[0][0])
                        : -1.0;
  double qa[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) qa[v] = c[v][0];
  nonpos = !(c[0][0] > 0.0) || !(pb > 0.0);
  if (nonpos) {   // Step 0: flatten the cell
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int l = 1; l < ML; ++l) c[v][l] = 0.0;
    smax = speed_of3(g, qa);
    return 0.0;
  }
  const double er = fmin(eps0, 0.5 * c[0][0]), ep = fmin(eps0, 0.5 * pb);
  double thr = 1.0, th = 1.0, sm = speed_of3(g, qa);
#pragma unroll 1
  for (int p = 0; p < NPT; ++p) {
    double ph[ML];
    load(p, ph);
    double q[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      double d = 0.0;
#pragma unroll
      for (int l = 1; l < ML; ++l) d = fma(c[v][l], ph[l], d);
      q[v] = c[v][0] + d;
    }
    if (q[0] < er) thr = fmin(thr, (c[0][0] - er) / (c[0][0] - q[0]));
    const double pt = g1 * (q[4] - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0]);
    if (pt < ep) th = fmin(th, (pb - ep) / (pb - pt));
    sm = fmax(sm, speed_of3(g, q));
  }
  if (thr < 1.0) {   // Step 2 again on the density-limited state
    th = thr;
#pragma unroll 1
    for (int p = 0; p < NPT; ++p) {
      double ph[ML];
      load(p, ph);
      double q[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double d = 0.0;
#pragma unroll
        for (int l = 1; l < ML; ++l) d = fma(c[v][l], ph[l], d);
        q[v] = c[v][0] + thr * d;
      }
      const double pt = g1 * (q[4] - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0]);
      if (pt < ep) th = fmin(th, thr * (pb - ep) / (pb - pt));
    }
  }
  th = fmax(th, 0.0);
  if (!(th < 1.0)) {
    smax = sm;
    return th;
  }
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int l = 1; l < ML; ++l) c[v][l] *= th;
  sm = speed_of3(g, qa);
#pragma unroll 1
  for (int p = 0; p < NPT; ++p) {
    double ph[ML];
    load(p, ph);
    double q[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      double acc = 0.0;
#pragma unroll
      for (int l = 0; l < ML; ++l) acc = fma(c[v][l], ph[l], acc);
      q[v] = acc;
    }
    sm = fmax(sm, speed_of3(g, q));
  }
  smax = sm;
  return th;
}

// ---------------------------------------------------------------- FP32 screens
// The mixed forms screen the moment and shock limiters in FP32.  With S_v =
// |c_v0| + sum_l |c_vl| max_p |phi_l(p)|, the FP32 value of variable v at any
// limiter point is within ~ML 2^-24 S_v of the exact one; kScreenTol = 1e-5
// leaves a margin of more than 10x.  A cell whose FP32 values clear the
// limiter's thresholds by that bound at every point is provably not limited
// in FP64 either; every other cell takes the FP64 path, so the decisions
// equal the FP64 form's.
constexpr float kScreenTol = 1e-5f;

template <int ML>
__device__ __forceinline__ void screen_state3(const double c[5][ML], const float* phimax, float cf[5][ML],
                                              float S[5]) {
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    float sv = 0.0f;
#pragma unroll
    for (int l = 0; l < ML; ++l) {
      cf[v][l] = opaque((float)c[v][l]);
      sv = fmaf(fabsf(cf[v][l]), phimax[l], sv);
    }
    S[v] = sv;
  }
}

// Sec. 3.1 screen: true when every point has rho > er and p > ep by more than
// the bound (theta = 1); smax is then the FP32 wave speed over the points.
template <int ML, int NPT, class LoadF>
__device__ __forceinline__ bool moment_screen3(const float cf[5][ML], const float S[5], float g, float er, float ep,
                                               const LoadF& loadf, float& smax) {
  const float g1 = g - 1.0f;
  float sm = 0.0f;
#pragma unroll 1
  for (int p = 0; p < NPT; ++p) {
    float ph[ML];
    loadf(p, ph);
    float q[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      float acc = cf[v][0];
#pragma unroll
      for (int l = 1; l < ML; ++l) acc = fmaf(cf[v][l], ph[l], acc);
      q[v] = acc;
    }
    if (!(q[0] > er * (1.0f + kScreenTol) + kScreenTol * S[0])) return false;
    const float ri = 1.0f / q[0];
    const float u = q[1] * ri, v = q[2] * ri, w = q[3] * ri;
    const float k2 = u * u + v * v + w * w;
    const float pp = g1 * (q[4] - 0.5f * q[0] * k2);
    const float B = S[4] + fabsf(u) * S[1] + fabsf(v) * S[2] + fabsf(w) * S[3] + 0.5f * k2 * S[0];
    if (!(pp > ep * (1.0f + kScreenTol) + kScreenTol * g1 * B)) return false;
    sm = fmaxf(sm, sqrtf(k2) + sqrtf(g * pp * ri));
  }
  smax = sm;
  return true;
}

// FP32 primitives (rho, u, v, w, p) of a state q with first-order bounds on
// their rounding, given bounds Sv on the error scale of each component
__device__ __forceinline__ void prim_bounds3(float g1, const float q[5], const float Sv[5], float wv[5], float ev[5]) {
  const float ri = 1.0f / q[0];
  const float u = q[1] * ri, v = q[2] * ri, w = q[3] * ri;
  const float k2 = u * u + v * v + w * w;
  wv[0] = q[0]; wv[1] = u; wv[2] = v; wv[3] = w; wv[4] = g1 * (q[4] - 0.5f * q[0] * k2);
  ev[0] = kScreenTol * Sv[0];
  ev[1] = kScreenTol * (Sv[1] + fabsf(u) * Sv[0]) * ri;
  ev[2] = kScreenTol * (Sv[2] + fabsf(v) * Sv[0]) * ri;
  ev[3] = kScreenTol * (Sv[3] + fabsf(w) * Sv[0]) * ri;
  ev[4] = kScreenTol * g1 * (Sv[4] + fabsf(u) * Sv[1] + fabsf(v) * Sv[2] + fabsf(w) * Sv[3] + 0.5f * k2 * Sv[0]);
}

// Sec. 4.1 bounds for the screen, in FP32: a lower bound hi on M = max(w_i +
// alpha, max_j w_j) and an upper bound lo on m = min(w_i - alpha, min_j w_j)
// from the cell average qb and the neighbour (or mirrored) averages given by
// nbr(k, qn) (false: no such neighbour, or a non-positive density)
template <int E, class Nbr>
__device__ __forceinline__ bool shock_bounds3(float g, float alpha, const float qb[5], const Nbr& nbr, float hi[5],
                                              float lo[5]) {
  const float g1 = g - 1.0f;
  float Sb[5], wb[5], eb[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) Sb[v] = fabsf(qb[v]);
  if (!(qb[0] > 0.0f)) return false;
  prim_bounds3(g1, qb, Sb, wb, eb);
  const float al = alpha * (1.0f - kScreenTol);
#pragma unroll
  for (int v = 0; v < 5; ++v) { hi[v] = wb[v] + al - eb[v]; lo[v] = wb[v] - al + eb[v]; }
#pragma unroll 1
  for (int k = 0; k < E; ++k) {
    float qn[5];
    if (!nbr(k, qn) || !(qn[0] > 0.0f)) continue;
    float Sn[5], wn[5], en[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) Sn[v] = fabsf(qn[v]);
    prim_bounds3(g1, qn, Sn, wn, en);
#pragma unroll
    for (int v = 0; v < 5; ++v) { hi[v] = fmaxf(hi[v], wn[v] - en[v]); lo[v] = fminf(lo[v], wn[v] + en[v]); }
  }
  return true;
}

// Sec. 4.1 screen: true when every point's primitives lie inside [lo, hi]
// (FP32 bounds inside the exact [m, M]) by more than their rounding bounds
// (theta = 1).
template <int ML, int NPT, class LoadF>
__device__ __forceinline__ bool shock_screen3(const float cf[5][ML], const float S[5], float g, const float hi[5],
                                              const float lo[5], const LoadF& loadf) {
  const float g1 = g - 1.0f;
#pragma unroll 1
  for (int p = 0; p < NPT; ++p) {
    float ph[ML];
    loadf(p, ph);
    float q[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      float acc = cf[v][0];
#pragma unroll
      for (int l = 1; l < ML; ++l) acc = fmaf(cf[v][l], ph[l], acc);
      q[v] = acc;
    }
    if (!(q[0] > 2.0f * kScreenTol * S[0])) return false;
    float wv[5], ev[5];
    prim_bounds3(g1, q, S, wv, ev);
#pragma unroll
    for (int c = 0; c < 5; ++c)
      if (!(wv[c] + ev[c] <= hi[c] && wv[c] - ev[c] >= lo[c])) return false;
  }
  return true;
}

// ---------------------------------------------------------------- normal flux
// n . F and its derivatives along n, for the face points, where only the
// normal component of F_T is needed: n . F(q) = (m . n, m (u . n) + p n,
// (E + p) u . n); the first and second derivatives follow flux3_d1 and
// flux3_d2 dotted with n.
template <typename T>
__device__ __forceinline__ void fluxn3(const P3T<T>& s, const T n[3], T F[5]) {
  const T un = s.u[0] * n[0] + s.u[1] * n[1] + s.u[2] * n[2];
  F[0] = s.q[1] * n[0] + s.q[2] * n[1] + s.q[3] * n[2];
#pragma unroll
  for (int e = 0; e < 3; ++e) F[1 + e] = s.q[1 + e] * un + s.p * n[e];
  F[4] = (s.q[4] + s.p) * un;
}

template <typename T>
__device__ __forceinline__ void fluxn3_d1(T g1, const P3T<T>& s, const T n[3], const T w[5], T F[5], T du[3], T& dp) {
#pragma unroll
  for (int d = 0; d < 3; ++d) du[d] = (w[1 + d] - s.u[d] * w[0]) * s.ri;
  const T k2 = s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2];
  dp = g1 * (w[4] - (s.u[0] * w[1] + s.u[1] * w[2] + s.u[2] * w[3]) + T(0.5) * k2 * w[0]);
  const T un = s.u[0] * n[0] + s.u[1] * n[1] + s.u[2] * n[2];
  const T dun = du[0] * n[0] + du[1] * n[1] + du[2] * n[2];
  F[0] = w[1] * n[0] + w[2] * n[1] + w[3] * n[2];
#pragma unroll
  for (int e = 0; e < 3; ++e) F[1 + e] = w[1 + e] * un + s.q[1 + e] * dun + dp * n[e];
  F[4] = (w[4] + dp) * un + (s.q[4] + s.p) * dun;
}

template <typename T>
__device__ __forceinline__ void fluxn3_d2(T g1, const P3T<T>& s, const T n[3], const T w[5], const T du[3], T dp,
                                          T F[5]) {
  T d2u[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) d2u[d] = T(-2) * w[0] * du[d] * s.ri;
  const T d2p = -g1 * ((w[1] * du[0] + w[2] * du[1] + w[3] * du[2]) +
                       T(0.5) * (s.q[1] * d2u[0] + s.q[2] * d2u[1] + s.q[3] * d2u[2]));
  const T un = s.u[0] * n[0] + s.u[1] * n[1] + s.u[2] * n[2];
  const T dun = du[0] * n[0] + du[1] * n[1] + du[2] * n[2];
  const T d2un = d2u[0] * n[0] + d2u[1] * n[1] + d2u[2] * n[2];
  F[0] = T(0);
#pragma unroll
  for (int e = 0; e < 3; ++e) F[1 + e] = T(2) * w[1 + e] * dun + s.q[1 + e] * d2un + d2p * n[e];
  F[4] = d2p * un + T(2) * (w[4] + dp) * dun + (s.q[4] + s.p) * d2un;
}

// q and n . F_T = n . (F + dt/2 F_t + dt^2/6 F_tt) at a point from the basis values
template <typename T, int ML>
__device__ __forceinline__ void ftn_point3(T g1, T c1, T c2, const T n[3], const T ph[ML], const T c[5][ML],
                                           const T Qt[5][ML], const T Qtt[5][ML], T q[5], T FTn[5]) {
  T qt[5], qtt[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    T acc = T(0), d1 = T(0), d2 = T(0);
#pragma unroll
    for (int l = 0; l < ML; ++l) {
      acc = fmaT(c[v][l], ph[l], acc);
      d1 = fmaT(Qt[v][l], ph[l], d1);
      d2 = fmaT(Qtt[v][l], ph[l], d2);
    }
    q[v] = acc; qt[v] = d1; qtt[v] = d2;
  }
  const P3T<T> s = make_p3<T>(g1, q);
  T F[5], F1[5], F2[5], F3[5], du[3], dp, eu[3], ep;
  fluxn3<T>(s, n, F);
  fluxn3_d1<T>(g1, s, n, qt, F1, du, dp);
  fluxn3_d2<T>(g1, s, n, qt, du, dp, F2);
  fluxn3_d1<T>(g1, s, n, qtt, F3, eu, ep);
#pragma unroll
  for (int v = 0; v < 5; ++v) FTn[v] = F[v] + c1 * F1[v] + c2 * (F2[v] + F3[v]);
}
