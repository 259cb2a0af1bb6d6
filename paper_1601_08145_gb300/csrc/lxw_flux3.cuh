// lxw_flux3.cuh -- device helpers of the 3D FP64 forms (hexahedra and
// tetrahedra): the Euler flux in three directions, its first and second
// directional derivatives (the Cauchy-Kovalevskaya terms of Sec. 2.2), the
// wave speed and the local Lax-Friedrichs speed.  Included inside each
// kernel file's anonymous namespace.
#pragma once

__device__ __forceinline__ double speed_of3(double g, const double q[5]) {
  if (!(q[0] > 0.0)) return 0.0;
  const double ri = 1.0 / q[0];
  const double u = q[1] * ri, v = q[2] * ri, w = q[3] * ri;
  const double k2 = u * u + v * v + w * w;
  const double p = (g - 1.0) * (q[4] - 0.5 * q[0] * k2);
  return sqrt(k2) + (p > 0.0 ? sqrt(g * p * ri) : 0.0);
}

// The local Lax-Friedrichs speed of a trace with explicitly rounded
// operations: both cells of a face evaluate it on the same two traces and
// must get the same value.
__device__ __forceinline__ double lf_speed3(double g, const double q[5]) {
  if (!(q[0] > 0.0)) return 0.0;
  const double ri = __drcp_rn(q[0]);
  const double u = __dmul_rn(q[1], ri), v = __dmul_rn(q[2], ri), w = __dmul_rn(q[3], ri);
  const double k2 = __dadd_rn(__dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)), __dmul_rn(w, w));
  const double p = __dmul_rn(g - 1.0, __dsub_rn(q[4], __dmul_rn(0.5, __dmul_rn(q[0], k2))));
  const double c = p > 0.0 ? __dsqrt_rn(__dmul_rn(__dmul_rn(g, p), ri)) : 0.0;
  return __dadd_rn(__dsqrt_rn(k2), c);
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
// Point state with its primitives.
struct P3 {
  double q[5];
  double ri, u[3], p;
};
__device__ __forceinline__ P3 make_p3(double g1, const double q[5]) {
  P3 s;
#pragma unroll
  for (int v = 0; v < 5; ++v) s.q[v] = q[v];
  s.ri = 1.0 / q[0];
#pragma unroll
  for (int d = 0; d < 3; ++d) s.u[d] = q[1 + d] * s.ri;
  s.p = g1 * (q[4] - 0.5 * (q[1] * s.u[0] + q[2] * s.u[1] + q[3] * s.u[2]));
  return s;
}

// F_d(q), d = 0, 1, 2
__device__ __forceinline__ void flux3(const P3& s, double F[3][5]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F[d][0] = s.q[1 + d];
#pragma unroll
    for (int e = 0; e < 3; ++e) F[d][1 + e] = s.q[1 + e] * s.u[d] + (e == d ? s.p : 0.0);
    F[d][4] = (s.q[4] + s.p) * s.u[d];
  }
}

// F'(q) w; also the primitive increments du (velocity) and dp along w
__device__ __forceinline__ void flux3_d1(double g1, const P3& s, const double w[5], double F[3][5], double du[3],
                                         double& dp) {
#pragma unroll
  for (int d = 0; d < 3; ++d) du[d] = (w[1 + d] - s.u[d] * w[0]) * s.ri;
  const double k2 = s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2];
  dp = g1 * (w[4] - (s.u[0] * w[1] + s.u[1] * w[2] + s.u[2] * w[3]) + 0.5 * k2 * w[0]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F[d][0] = w[1 + d];
#pragma unroll
    for (int e = 0; e < 3; ++e) F[d][1 + e] = w[1 + e] * s.u[d] + s.q[1 + e] * du[d] + (e == d ? dp : 0.0);
    F[d][4] = (w[4] + dp) * s.u[d] + (s.q[4] + s.p) * du[d];
  }
}

// F''(q)(w, w) from the increments of flux3_d1: along q + t w the density
// and momentum are linear, so u'' = -2 w_rho u' / rho and
// p'' = -(g-1)(m' . u' + m . u'' / 2)
__device__ __forceinline__ void flux3_d2(double g1, const P3& s, const double w[5], const double du[3], double dp,
                                         double F[3][5]) {
  double d2u[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) d2u[d] = -2.0 * w[0] * du[d] * s.ri;
  const double d2p = -g1 * ((w[1] * du[0] + w[2] * du[1] + w[3] * du[2]) +
                            0.5 * (s.q[1] * d2u[0] + s.q[2] * d2u[1] + s.q[3] * d2u[2]));
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F[d][0] = 0.0;
#pragma unroll
    for (int e = 0; e < 3; ++e) F[d][1 + e] = 2.0 * w[1 + e] * du[d] + s.q[1 + e] * d2u[d] + (e == d ? d2p : 0.0);
    F[d][4] = d2p * s.u[d] + 2.0 * (w[4] + dp) * du[d] + (s.q[4] + s.p) * d2u[d];
  }
}

