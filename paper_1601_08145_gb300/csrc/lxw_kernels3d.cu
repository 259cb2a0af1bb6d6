// lxw_kernels3d.cu -- sm_103a kernels of one LxW-DG step on 3D Cartesian
// meshes (hexahedra), the extension the paper says carries over directly
// (end of Sec. 3.3; the 3D Euler equations of Sec. 1.1 with the third flux
// H).  Two forms: FP64 throughout, and mixed (Args3::ck_fp32): the CK kernel
// and the face point loop in FP32, FP32 screens in the moment and shock
// limiters, the state, averages, f^LxF, Steps 4-5 and every limiter
// decision in FP64.
//
// One thread owns one cell, as in the 2D FP64 form; state Q[N][5][ML]
// (rho, rho u, rho v, rho w, E), modes ordered by total degree, then the x
// exponent descending, then the y exponent descending.  Phases (kernel
// boundaries carry the grid-wide dependencies):
//   k3_moment  Sec. 3.1 moment limiter + max |u| + c -> atomicMax
//   k3_ck      Sec. 2.2-2.3 CK flux (q_t, q_tt carried as modes through the
//              weighted differentiation tables), volume integral, traces
//   k3_face    Sec. 3.3 Step 3 on six faces (LLF with the local speed,
//              f^LxW, f^LxF, face integral) and Steps 4-5 (Lambda, 63
//              corners, mu) per cell
//   k3_update  Step 6: theta = min of both proposals, averages
//   k3_shock   Sec. 4.1 on (rho, u, v, w, p) with the six face neighbours
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "lxw_internal3d.h"

namespace lxw {
namespace {

__constant__ Tables3 c_tab3[2];    // degree 1, degree 2
__constant__ Tables3F c_tab3f[2];  // their FP32 copies (the mixed form's CK kernel)

#include "lxw_flux3.cuh"

template <typename T>
__device__ __forceinline__ const Tables3Of<T>& tab3(int deg);
template <>
__device__ __forceinline__ const Tables3Of<double>& tab3<double>(int deg) { return c_tab3[deg - 1]; }
template <>
__device__ __forceinline__ const Tables3Of<float>& tab3<float>(int deg) { return c_tab3f[deg - 1]; }


__device__ __forceinline__ double step_dt3(const Work3& w, const Mesh3& m, const Args3& a) {
  const double s = __longlong_as_double((long long)*w.smax);
  return a.dt_in > 0.0 ? a.dt_in : a.cfl * m.hmin / s;
}

// ------------------------------------------------------------ k3_reset
__global__ void k3_reset(Work3 w, int want_diag) {
  if (threadIdx.x == 0) {
    *w.smax = 0ull;
    *w.status = 0u;
  }
  if (want_diag && threadIdx.x < 5) w.diag->sum[threadIdx.x] = 0.0;
  if (want_diag && threadIdx.x == 0) {
    w.diag->minr = w.diag->minp = ~0ull;
    w.diag->nmom = w.diag->nface = w.diag->nsc = 0ull;
  }
}

// ------------------------------------------------------------ k3_moment
// Sec. 3.1 Steps 0-2 (Lemma 1's secant), then |u| + c of the limited state at
// every point and of the average, block max -> atomicMax.
template <int DEG, int ML, int N1>
__global__ void __launch_bounds__(128) k3_moment(const Mesh3 m, const Work3 w, double* __restrict__ Q, const Args3 a) {
  constexpr int NQ = N1 * N1 * N1, NF = N1 * N1, NPT = NQ + 6 * NF;
  const Tables3& t = c_tab3[DEG - 1];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double smax = 0.0;
  if (i < m.N) {
    double* Qi = Q + (size_t)i * 5 * ML;
    double c[5][ML];
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int l = 0; l < ML; ++l) c[v][l] = Qi[v * ML + l];
    {   // the Euler flux of the average, read by the face kernel for this cell and its neighbours
      double qa[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) qa[v] = c[v][0];
      const P3 sa = make_p3(a.gamma - 1.0, qa);
      double Fa[3][5];
      flux3(sa, Fa);
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 5; ++v) w.fbar[(size_t)(d * 5 + v) * m.N + i] = Fa[d][v];
    }
    auto load = [&](int p, double ph[ML]) {
#pragma unroll
      for (int l = 0; l < ML; ++l) ph[l] = t.phi[p][l];
    };
    bool screened = false;
    if (a.ck_fp32 && c[0][0] > 0.0) {   // mixed form: the FP32 screen clears unlimited cells
      const double pb = (a.gamma - 1.0) * (c[4][0] - 0.5 * (c[1][0] * c[1][0] + c[2][0] * c[2][0] + c[3][0] * c[3][0]) / c[0][0]);
      if (pb > 0.0) {
        const Tables3Of<float>& tf = tab3<float>(DEG);
        float cf[5][ML], S[5], smf;
        screen_state3<ML>(c, tf.phimax, cf, S);
        auto loadf = [&](int p, float ph[ML]) {
#pragma unroll
          for (int l = 0; l < ML; ++l) ph[l] = tf.phi[p][l];
        };
        if (moment_screen3<ML, NPT>(cf, S, (float)a.gamma, (float)fmin(a.eps0, 0.5 * c[0][0]), (float)fmin(a.eps0, 0.5 * pb),
                                    loadf, smf)) {
          double qa[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) qa[v] = c[v][0];
          smax = fmax((double)smf, speed_of3(a.gamma, qa));
          screened = true;
        }
      }
    }
    bool nonpos = false;
    const double th = screened ? 1.0 : moment_cell3<ML, NPT>(c, a.gamma, a.eps0, load, smax, nonpos);
    if (nonpos) atomicOr(w.status, (unsigned)LXW_ST_NONPOSITIVE);
    if (th < 1.0) {
#pragma unroll
      for (int v = 0; v < 5; ++v)
#pragma unroll
        for (int l = 1; l < ML; ++l) Qi[v * ML + l] = c[v][l];
      if (a.want_diag) atomicAdd(&w.diag->nmom, 1ull);
    }
  }
  block_max3(smax, w.smax);
}

// ------------------------------------------------------------ k3_ck
// Sec. 2.2-2.3: q_t = -div F^h and q_tt = -div F_t^h lie in the modal space
// (degree deg - 1), so they are carried as modal coefficients Qt, Qtt,
// accumulated at the interior points with the weighted differentiation
// tables (the same values as projecting the flux and differentiating the
// expansion); F_t = F'(q) q_t, F_tt = F''(q)(q_t, q_t) + F'(q) q_tt, F_T =
// F + dt/2 F_t + dt^2/6 F_tt at every point; the volume integral is added to
// the higher moments in place, the face points store q and n_out . F_T.
// T = double: the FP64 form; T = float: the mixed form's FP32 kernel (the
// state stays FP64 and the volume term is added to it in FP64; the traces
// are stored in T, the face kernel of the same form reads them in T).
template <typename T, int DEG, int ML, int N1>
__global__ void __launch_bounds__(128) k3_ck(const Mesh3 m, const Work3 w, double* __restrict__ Q, const Args3 a) {
  constexpr int NQ = N1 * N1 * N1, NF = N1 * N1, NPT = NQ + 6 * NF;
  constexpr bool F64 = sizeof(T) == 8;
  const Tables3Of<T>& t = tab3<T>(DEG);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const int N = m.N;
  const T g1 = opaque(T(a.gamma - 1.0));
  const double dtd = step_dt3(w, m, a);
  const T dt = T(dtd);
  const T c1 = opaque(T(0.5 * dtd)), c2 = opaque(T(dtd * dtd / 6.0));
  const T sd[3] = {opaque(T(2.0 / m.h[0])), opaque(T(2.0 / m.h[1])), opaque(T(2.0 / m.h[2]))};
  const T avh[3] = {opaque(T(m.vol / m.h[0])), opaque(T(m.vol / m.h[1])), opaque(T(m.vol / m.h[2]))};
  double* Qi = Q + (size_t)i * 5 * ML;
  // FP32 form: read the coefficients once (a volatile view) and pin the
  // converted values, so that the compiler keeps (or spills) them instead of
  // reloading or re-converting the FP64 state at every use (conversions run
  // on the FP64 pipe)
  T c[5][ML];
  const volatile double* Qv = Qi;
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) {
      if constexpr (F64) c[v][l] = Qi[v * ML + l];
      else c[v][l] = opaque(T(Qv[v * ML + l]));
    }
  // pass 1: Qt
  T Qt[5][ML];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) Qt[v][l] = T(0);
#pragma unroll 1
  for (int k = 0; k < NQ; ++k) {
    T q[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      T acc = T(0);
#pragma unroll
      for (int l = 0; l < ML; ++l) acc = fmaT(c[v][l], t.phi[k][l], acc);
      q[v] = acc;
    }
    const P3T<T> s = make_p3<T>(g1, q);
    T F[3][5];
    flux3<T>(s, F);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const T f0 = sd[0] * F[0][v], f1 = sd[1] * F[1][v], f2 = sd[2] * F[2][v];
#pragma unroll
      for (int l = 0; l < ML; ++l)
        Qt[v][l] = fmaT(-f2, t.W[2][k][l], fmaT(-f1, t.W[1][k][l], fmaT(-f0, t.W[0][k][l], Qt[v][l])));
    }
  }
  // pass 2: Qtt
  T Qtt[5][ML];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) Qtt[v][l] = T(0);
#pragma unroll 1
  for (int k = 0; k < NQ; ++k) {
    T q[5], qt[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      T acc = T(0), d1 = T(0);
#pragma unroll
      for (int l = 0; l < ML; ++l) {
        acc = fmaT(c[v][l], t.phi[k][l], acc);
        d1 = fmaT(Qt[v][l], t.phi[k][l], d1);
      }
      q[v] = acc; qt[v] = d1;
    }
    const P3T<T> s = make_p3<T>(g1, q);
    T F1[3][5], du[3], dp;
    flux3_d1<T>(g1, s, qt, F1, du, dp);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const T f0 = sd[0] * F1[0][v], f1 = sd[1] * F1[1][v], f2 = sd[2] * F1[2][v];
#pragma unroll
      for (int l = 0; l < ML; ++l)
        Qtt[v][l] = fmaT(-f2, t.W[2][k][l], fmaT(-f1, t.W[1][k][l], fmaT(-f0, t.W[0][k][l], Qtt[v][l])));
    }
  }
  // pass 3a: F_T at the interior points -> volume integral of the higher moments
  T Vv[5][ML];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) Vv[v][l] = T(0);
#pragma unroll 1
  for (int p = 0; p < NQ; ++p) {
    T q[5], qt[5], qtt[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      T acc = T(0), d1 = T(0), d2 = T(0);
#pragma unroll
      for (int l = 0; l < ML; ++l) {
        const T ph = t.phi[p][l];
        acc = fmaT(c[v][l], ph, acc);
        d1 = fmaT(Qt[v][l], ph, d1);
        d2 = fmaT(Qtt[v][l], ph, d2);
      }
      q[v] = acc; qt[v] = d1; qtt[v] = d2;
    }
    const P3T<T> s = make_p3<T>(g1, q);
    T F[3][5], FT[3][5];
    flux3<T>(s, F);
    {
      T F1[3][5], du[3], dp;
      flux3_d1<T>(g1, s, qt, F1, du, dp);
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 5; ++v) FT[d][v] = F[d][v] + c1 * F1[d][v];
      flux3_d2<T>(g1, s, qt, du, dp, F1);
      T F3[3][5], eu[3], ep;
      flux3_d1<T>(g1, s, qtt, F3, eu, ep);
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 5; ++v) FT[d][v] += c2 * (F1[d][v] + F3[d][v]);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const T f0 = t.qw[p] * sd[0] * FT[0][v], f1 = t.qw[p] * sd[1] * FT[1][v], f2 = t.qw[p] * sd[2] * FT[2][v];
#pragma unroll
      for (int l = 1; l < ML; ++l)
        Vv[v][l] = fmaT(f0, t.dref[0][p][l], fmaT(f1, t.dref[1][p][l], fmaT(f2, t.dref[2][p][l], Vv[v][l])));
    }
  }
  // pass 3b: q and n_out . F_T (n scaled by the face area) at the face points
#pragma unroll 1
  for (int p = NQ; p < NPT; ++p) {
    const int k = (p - NQ) / NF, pe = (p - NQ) - k * NF, d = k >> 1;
    T nv[3] = {T(0), T(0), T(0)};
    nv[d] = (k & 1) ? avh[d] : -avh[d];   // outward normal times the face area
    T ph[ML], q[5], FTn[5];
#pragma unroll
    for (int l = 0; l < ML; ++l) ph[l] = t.phi[p][l];
    ftn_point3<T, ML>(g1, c1, c2, nv, ph, c, Qt, Qtt, q, FTn);
    T* tr = reinterpret_cast<T*>(w.trace) + ((size_t)(k * NF + pe) * 10) * N + i;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      tr[(size_t)v * N] = q[v];
      tr[(size_t)(5 + v) * N] = FTn[v];
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int l = 1; l < ML; ++l) {
      if constexpr (F64) Qi[v * ML + l] = c[v][l] + dt * Vv[v][l];
      else Qi[v * ML + l] += dtd * double(Vv[v][l]);
    }
}

// ------------------------------------------------------------ k3_face
// Sec. 3.3 Step 3 on the six faces, seen from each cell: both cells of a
// face take its points in the same order and the same explicitly rounded
// operations on negated operands, so their LLF values, f^LxW and f^LxF are
// exact negatives.  Face integral of the higher moments; Steps 4-5: Gamma,
// the density Lambda shared by the negative faces, the Lax-Friedrichs
// state, mu over the 63 corners of the box of proposals.
// T is the arithmetic of the point loop (the traces, the LLF values, f^LxW
// and the face integral: FP32 in the mixed form); the averages, f^LxF and
// Steps 4-5 are FP64 in both forms.
template <typename T, int DEG, int ML, int N1>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1) k3_face(const Mesh3 m, const Work3 w, double* __restrict__ Q, const Args3 a) {
  constexpr int NQ = N1 * N1 * N1, NF = N1 * N1;
  const Tables3Of<T>& t = tab3<T>(DEG);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const int N = m.N;
  const double g = a.gamma, g1 = g - 1.0;
  const T gT = T(g);
  const double s = __longlong_as_double((long long)*w.smax);
  const double dt = step_dt3(w, m, a);
  const T* trb = reinterpret_cast<const T*>(w.trace);
  double* Qi = Q + (size_t)i * 5 * ML;
  double qb[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) qb[v] = Qi[v * ML];
  T Ei[5][ML];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) Ei[v][l] = T(0);
  double fW[6][5], fF[6][5];
#pragma unroll 1
  for (int k = 0; k < 6; ++k) {
    const int j = m.nbr[k * N + i], d = k >> 1, kj = k ^ 1;
    const double an = (k & 1 ? 1.0 : -1.0) * m.vol / m.h[d];
    const double area = fabs(an);
    const double hs = 0.5 * s * area;
    // neighbour (or exterior) average: reflection flips the normal momentum
    double qn[5];
    if (j >= 0) {
      const double* Qj = Q + (size_t)j * 5 * ML;
#pragma unroll
      for (int v = 0; v < 5; ++v) qn[v] = Qj[v * ML];
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) qn[v] = qb[v];
      if (-1 - j == LXW_BC_REFLECT) qn[1 + d] = -qn[1 + d];
    }
    {
      // the averages' fluxes along axis d: this cell's and an interior neighbour's
      // from the moment kernel, a wall's mirrored state computed here
      double Fbd[5], Fnd[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) Fbd[v] = w.fbar[(size_t)(d * 5 + v) * N + i];
      if (j >= 0) {
#pragma unroll
        for (int v = 0; v < 5; ++v) Fnd[v] = w.fbar[(size_t)(d * 5 + v) * N + j];
      } else if (-1 - j == LXW_BC_REFLECT) {
        const P3 sn = make_p3(g1, qn);
        double Fn[3][5];
        flux3(sn, Fn);
#pragma unroll
        for (int v = 0; v < 5; ++v) Fnd[v] = Fn[d][v];
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) Fnd[v] = Fbd[v];
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double ai = __dmul_rn(an, Fbd[v]), ak = __dmul_rn(an, Fnd[v]);
        fF[k][v] = __fma_rn(-hs, __dsub_rn(qn[v], qb[v]), __dmul_rn(0.5, __dadd_rn(ai, ak)));
      }
    }
    T fWk[5] = {T(0), T(0), T(0), T(0), T(0)};
    const T hsT = T(hs), sT = T(s), areaT = T(area);
#pragma unroll 1
    for (int p = 0; p < NF; ++p) {
      const T* tr = trb + ((size_t)(k * NF + p) * 10) * N + i;
      T qi[5], Fi[5], qx[5], Fx[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) { qi[v] = tr[(size_t)v * N]; Fi[v] = tr[(size_t)(5 + v) * N]; }
      if (j >= 0) {
        const T* tj = trb + ((size_t)(kj * NF + p) * 10) * N + j;
#pragma unroll
        for (int v = 0; v < 5; ++v) { qx[v] = tj[(size_t)v * N]; Fx[v] = -tj[(size_t)(5 + v) * N]; }
      } else if (-1 - j == LXW_BC_REFLECT) {
        // exterior R q, and n . F_T(R q) = -R (n . F_T(q)) (the Euler flux's mirror symmetry)
#pragma unroll
        for (int v = 0; v < 5; ++v) { qx[v] = qi[v]; Fx[v] = -Fi[v]; }
        qx[1 + d] = -qi[1 + d];
        Fx[1 + d] = Fi[1 + d];
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) { qx[v] = qi[v]; Fx[v] = Fi[v]; }
      }
      // dissipation speed: the local speed of the two traces, at most s
      const T hp = a.llf_global ? hsT : T(0.5) * fminT(sT, fmaxT(lf_speed3<T>(gT, qi), lf_speed3<T>(gT, qx))) * areaT;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const T fs = rn_fma(-hp, rn_sub(qx[v], qi[v]), rn_mul(T(0.5), rn_add(Fi[v], Fx[v])));
        fWk[v] = rn_fma(t.fw[p], fs, fWk[v]);
        const T hw = t.fw[p] * fs;
#pragma unroll
        for (int l = 1; l < ML; ++l) Ei[v][l] = fmaT(hw, t.phi[NQ + k * NF + p][l], Ei[v][l]);
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) fW[k][v] = double(fWk[v]);
  }
  const double dta = dt / m.vol;
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int l = 1; l < ML; ++l) Qi[v * ML + l] -= dta * double(Ei[v][l]);

  // Steps 4-5
  double Gam0 = m.vol / dt * qb[0];
#pragma unroll
  for (int k = 0; k < 6; ++k) Gam0 -= fF[k][0];
  if (Gam0 < 0.0) atomicOr(w.status, (unsigned)LXW_ST_CFL);
  double neg = 0.0;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double df = fF[k][0] - fW[k][0];
    if (df < 0.0) neg += df;
  }
  double ql[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) acc += fF[k][v];
    ql[v] = qb[v] - dta * acc;
  }
  const double er = fmax(fmin(a.eps0, 0.5 * ql[0]), 0.0);
  double lneg = 1.0;
  if (neg < 0.0) lneg = fmin(1.0, fmax(0.0, (Gam0 - m.vol / dt * er) / (-neg)));
  double lam[6], dq[6][5];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    lam[k] = (fF[k][0] - fW[k][0]) < 0.0 ? lneg : 1.0;
#pragma unroll
    for (int v = 0; v < 5; ++v) dq[k][v] = dta * lam[k] * (fF[k][v] - fW[k][v]);
  }
  const double pl =
      ql[0] > 0.0 ? g1 * (ql[4] - 0.5 * (ql[1] * ql[1] + ql[2] * ql[2] + ql[3] * ql[3]) / ql[0]) : -1.0;
  double mmin[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) mmin[k] = 1.0;
  if (!(ql[0] > 0.0) || !(pl > 0.0)) {
#pragma unroll
    for (int k = 0; k < 6; ++k) mmin[k] = 0.0;
  } else {
    const double kap = fmin(a.eps0, 0.5 * pl) / g1;
    const double h0 = ql[0] * ql[4] - 0.5 * (ql[1] * ql[1] + ql[2] * ql[2] + ql[3] * ql[3]) - kap * ql[0];
    // every corner ql + dd has |dd_v| <= D_v = sum_k |dq_kv|, so h(ql + dd) >= h0
    // - (|rho| D_E + |E - kappa| D_rho + |m| . D_m) - (D_rho D_E + |D_m|^2 / 2):
    // when that bound (and rho - D_rho) clears zero by more than the rounding,
    // every corner is positive and every mu is 1 without the corner loop
    double D[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
      for (int v = 0; v < 5; ++v) D[v] += fabs(dq[k][v]);
    const double lin = fabs(ql[0]) * D[4] + fabs(ql[4] - kap) * D[0] + fabs(ql[1]) * D[1] + fabs(ql[2]) * D[2] +
                       fabs(ql[3]) * D[3];
    const double quad = D[0] * D[4] + 0.5 * (D[1] * D[1] + D[2] * D[2] + D[3] * D[3]);
    const double scale = fabs(ql[0] * ql[4]) + 0.5 * (ql[1] * ql[1] + ql[2] * ql[2] + ql[3] * ql[3]) +
                         fabs(kap * ql[0]) + lin + quad;
    const bool all_pos = ql[0] - D[0] > 1e-12 * ql[0] && h0 - lin - quad > 1e-12 * scale;
#pragma unroll 1
    for (int cm = all_pos ? 64 : 1; cm < 64; ++cm) {
      double dd[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if ((cm >> k) & 1)
#pragma unroll
          for (int v = 0; v < 5; ++v) dd[v] += dq[k][v];
      // h(mu) = rho E - |m|^2 / 2 - kappa rho along ql + mu dd
      const double h1 = ql[0] * dd[4] + dd[0] * ql[4] - (ql[1] * dd[1] + ql[2] * dd[2] + ql[3] * dd[3]) - kap * dd[0];
      const double h2 = dd[0] * dd[4] - 0.5 * (dd[1] * dd[1] + dd[2] * dd[2] + dd[3] * dd[3]);
      double mu = 1.0;
      if (!(ql[0] + dd[0] > 0.0) || h0 + h1 + h2 < 0.0) {
        const double disc = fmax(h1 * h1 - 4.0 * h0 * h2, 0.0);
        const double den = -h1 + sqrt(disc);
        mu = den > 0.0 ? fmin(1.0, fmax(0.0, 2.0 * h0 / den)) : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if ((cm >> k) & 1) mmin[k] = fmin(mmin[k], mu);
    }
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    w.prop[k * N + i] = lam[k] * mmin[k];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      w.flux[(size_t)(k * 10 + v) * N + i] = fW[k][v];
      w.flux[(size_t)(k * 10 + 5 + v) * N + i] = fF[k][v];
    }
  }
}

// ------------------------------------------------------------ k3_update
// Sec. 3.3 Step 6: theta of a face = min of the two cells' proposals;
// blended update of the averages.
template <int ML>
__global__ void __launch_bounds__(128) k3_update(const Mesh3 m, const Work3 w, double* __restrict__ Q, const Args3 a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const int N = m.N;
  const double dt = step_dt3(w, m, a);
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int j = m.nbr[k * N + i];
    double th = w.prop[k * N + i];
    if (j >= 0) th = fmin(th, w.prop[(k ^ 1) * N + j]);
    if (a.theta_face) a.theta_face[(size_t)i * 6 + k] = th;
    // count each face once: from its + side, or from the cell of a boundary face
    if (a.want_diag && th < 1.0 && (j < 0 || (k & 1))) atomicAdd(&w.diag->nface, 1ull);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double fw = w.flux[(size_t)(k * 10 + v) * N + i], ff = w.flux[(size_t)(k * 10 + 5 + v) * N + i];
      acc[v] += th * fw + (1.0 - th) * ff;
    }
  }
  double* Qi = Q + (size_t)i * 5 * ML;
  const double dta = dt / m.vol;
#pragma unroll
  for (int v = 0; v < 5; ++v) Qi[v * ML] -= dta * acc[v];
}

// ------------------------------------------------------------ k3_shock
// Sec. 4.1 on (rho, u, v, w, p): M = max(w_i + alpha, max_j w_j), m =
// min(w_i - alpha, min_j w_j) over the six face neighbours (a wall's
// exterior: the mirrored average), theta = min(1, (M - w_i)/(max_pts w -
// w_i), (w_i - m)/(w_i - min_pts w)) over the primitives, alpha = alpha0
// dx^1.5 with dx = |K|^(1/3).
template <int DEG, int ML, int N1>
__global__ void __launch_bounds__(128) k3_shock(const Mesh3 m, const Work3 w, double* __restrict__ Q, const Args3 a) {
  constexpr int NQ = N1 * N1 * N1, NF = N1 * N1, NPT = NQ + 6 * NF;
  const Tables3& t = c_tab3[DEG - 1];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const int N = m.N;
  const double g1 = a.gamma - 1.0;
  double* Qi = Q + (size_t)i * 5 * ML;
  double c[5][ML];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) c[v][l] = Qi[v * ML + l];
  auto prim = [&](const double q[5], double wv[5]) {
    const double ri = 1.0 / q[0];
    wv[0] = q[0]; wv[1] = q[1] * ri; wv[2] = q[2] * ri; wv[3] = q[3] * ri;
    wv[4] = g1 * (q[4] - 0.5 * (q[1] * wv[1] + q[2] * wv[2] + q[3] * wv[3]));
  };
  double th = 1.0;
  if (!(c[0][0] > 0.0)) {
    th = 0.0;
  } else {
    if (a.ck_fp32) {   // mixed form: FP32 bounds and points clear cells well inside [m, M]
      const Tables3Of<float>& tf = tab3<float>(DEG);
      float cf[5][ML], S[5], qbf[5], hi[5], lo[5];
      screen_state3<ML>(c, tf.phimax, cf, S);
#pragma unroll
      for (int v = 0; v < 5; ++v) qbf[v] = cf[v][0];
      auto nbrf = [&](int k, float qn[5]) -> bool {
        const int j = m.nbr[k * N + i];
        if (j >= 0) {
          const double* Qj = Q + (size_t)j * 5 * ML;
#pragma unroll
          for (int v = 0; v < 5; ++v) qn[v] = (float)Qj[v * ML];
        } else {
#pragma unroll
          for (int v = 0; v < 5; ++v) qn[v] = qbf[v];
          if (-1 - j == LXW_BC_REFLECT) qn[1 + (k >> 1)] = -qn[1 + (k >> 1)];
        }
        return true;
      };
      auto loadf = [&](int p, float ph[ML]) {
#pragma unroll
        for (int l = 0; l < ML; ++l) ph[l] = tf.phi[p][l];
      };
      const float alf = (float)a.alpha0 * powf(cbrtf((float)m.vol), 1.5f);
      if (shock_bounds3<6>((float)a.gamma, alf, qbf, nbrf, hi, lo) &&
          shock_screen3<ML, NPT>(cf, S, (float)a.gamma, hi, lo, loadf))
        return;
    }
    double qb[5], wb[5], Mx[5], Mn[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qb[v] = c[v][0];
    prim(qb, wb);
    const double al = a.alpha0 * pow(cbrt(m.vol), 1.5);
#pragma unroll
    for (int v = 0; v < 5; ++v) { Mx[v] = wb[v] + al; Mn[v] = wb[v] - al; }
#pragma unroll 1
    for (int k = 0; k < 6; ++k) {
      const int j = m.nbr[k * N + i];
      double qn[5], wn[5];
      if (j >= 0) {
        const double* Qj = Q + (size_t)j * 5 * ML;
#pragma unroll
        for (int v = 0; v < 5; ++v) qn[v] = Qj[v * ML];
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) qn[v] = qb[v];
        if (-1 - j == LXW_BC_REFLECT) qn[1 + (k >> 1)] = -qn[1 + (k >> 1)];
      }
      if (!(qn[0] > 0.0)) continue;
      prim(qn, wn);
#pragma unroll
      for (int v = 0; v < 5; ++v) { Mx[v] = fmax(Mx[v], wn[v]); Mn[v] = fmin(Mn[v], wn[v]); }
    }
    double hx[5], hn[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) { hx[v] = -1e300; hn[v] = 1e300; }
    bool bad = false;
#pragma unroll 1
    for (int p = 0; p < NPT; ++p) {
      double q[5], wp[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double acc = 0.0;
#pragma unroll
        for (int l = 0; l < ML; ++l) acc = fma(c[v][l], t.phi[p][l], acc);
        q[v] = acc;
      }
      if (!(q[0] > 0.0)) { bad = true; break; }
      prim(q, wp);
#pragma unroll
      for (int v = 0; v < 5; ++v) { hx[v] = fmax(hx[v], wp[v]); hn[v] = fmin(hn[v], wp[v]); }
    }
    if (bad) {
      th = 0.0;
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        if (hx[v] > wb[v]) th = fmin(th, (Mx[v] - wb[v]) / (hx[v] - wb[v]));
        if (hn[v] < wb[v]) th = fmin(th, (wb[v] - Mn[v]) / (wb[v] - hn[v]));
      }
      th = fmax(th, 0.0);
    }
  }
  if (th < 1.0) {
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int l = 1; l < ML; ++l) Qi[v * ML + l] = th * c[v][l];
    if (a.want_diag) atomicAdd(&w.diag->nsc, 1ull);
  }
}

// ------------------------------------------------------------ k3_diag
// Totals |K| Q^(1) and minimum density / pressure of the averages; warp
// reductions first, one atomic per warp and quantity.
template <int ML>
__global__ void __launch_bounds__(256) k3_diag(const Mesh3 m, const Work3 w, const double* __restrict__ Q, double gamma) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool on = i < m.N;
  auto ob = [](double x) {   // order-preserving bits
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
  };
  double q[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  unsigned long long br = ~0ull, bp = ~0ull;
  bool nan = false;
  if (on) {
    const double* Qi = Q + (size_t)i * 5 * ML;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      q[v] = Qi[v * ML];
      nan = nan || !isfinite(q[v]);
    }
    const double p = (gamma - 1.0) * (q[4] - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0]);
    br = ob(q[0]);
    bp = ob(p);
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] *= m.vol;
  }
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] += __shfl_down_sync(0xffffffffu, q[v], o);
    const unsigned long long r = __shfl_down_sync(0xffffffffu, br, o), pp = __shfl_down_sync(0xffffffffu, bp, o);
    br = r < br ? r : br;
    bp = pp < bp ? pp : bp;
  }
  if (__any_sync(0xffffffffu, nan) && (threadIdx.x & 31) == 0) atomicOr(w.status, (unsigned)LXW_ST_NAN);
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int v = 0; v < 5; ++v) atomicAdd(&w.diag->sum[v], q[v]);
    atomicMin(&w.diag->minr, br);
    atomicMin(&w.diag->minp, bp);
  }
}

// ------------------------------------------------------------ k3_project
template <int ML>
__global__ void k3_project(int N, int NPJ, double gamma, const double* __restrict__ jw, const double* __restrict__ jphi,
                           const double* __restrict__ prim, double* __restrict__ Q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double acc[5][ML];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) acc[v][l] = 0.0;
  for (int p = 0; p < NPJ; ++p) {
    const double* wv = prim + ((size_t)i * NPJ + p) * 5;
    const double r = wv[0], u = wv[1], v = wv[2], ww = wv[3];
    const double q[5] = {r, r * u, r * v, r * ww, wv[4] / (gamma - 1.0) + 0.5 * r * (u * u + v * v + ww * ww)};
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int l = 0; l < ML; ++l) acc[c][l] = fma(jw[p] * q[c], jphi[p * ML + l], acc[c][l]);
  }
  double* Qi = Q + (size_t)i * 5 * ML;
#pragma unroll
  for (int c = 0; c < 5; ++c)
#pragma unroll
    for (int l = 0; l < ML; ++l) Qi[c * ML + l] = acc[c][l];
}

template <int DEG, int ML, int N1>
int step3_impl(const Mesh3& m, const Work3& w, double* Q, const Args3& a, cudaStream_t st, int block, void** events,
               int upto) {
  const int grid = (m.N + block - 1) / block;
  int ne = 0;
  auto mark = [&]() { if (events) cudaEventRecord((cudaEvent_t)events[ne++], st); };
  auto ok = [&]() { return cudaGetLastError() == cudaSuccess ? 0 : -1; };
  k3_reset<<<1, 32, 0, st>>>(w, a.want_diag);
  mark();
  k3_moment<DEG, ML, N1><<<grid, block, 0, st>>>(m, w, Q, a);
  mark();
  if (upto < 2) return ok();
  if (a.ck_fp32) k3_ck<float, DEG, ML, N1><<<grid, block, 0, st>>>(m, w, Q, a);
  else k3_ck<double, DEG, ML, N1><<<grid, block, 0, st>>>(m, w, Q, a);
  mark();
  if (upto < 3) return ok();
  if (a.ck_fp32) k3_face<float, DEG, ML, N1><<<grid, block, 0, st>>>(m, w, Q, a);
  else k3_face<double, DEG, ML, N1><<<grid, block, 0, st>>>(m, w, Q, a);
  mark();
  if (upto < 4) return ok();
  k3_update<ML><<<grid, block, 0, st>>>(m, w, Q, a);
  mark();
  if (upto < 5) return ok();
  if (a.shock_limiter) k3_shock<DEG, ML, N1><<<grid, block, 0, st>>>(m, w, Q, a);
  mark();
  if (a.want_diag) k3_diag<ML><<<(m.N + 255) / 256, 256, 0, st>>>(m, w, Q, a.gamma);
  return ok();
}

}  // namespace

int upload_tables3(int deg, const Tables3& t) {
  if (deg < 1 || deg > 2) return -1;
  Tables3F f;
  const double* src = &t.qw[0];
  float* dst = &f.qw[0];
  static_assert(sizeof(Tables3) == 2 * sizeof(Tables3F), "tables hold doubles only");
  for (size_t k = 0; k < sizeof(Tables3) / sizeof(double); ++k) dst[k] = (float)src[k];
  if (cudaMemcpyToSymbol(c_tab3, &t, sizeof(Tables3), sizeof(Tables3) * (deg - 1)) != cudaSuccess) return -1;
  return cudaMemcpyToSymbol(c_tab3f, &f, sizeof(Tables3F), sizeof(Tables3F) * (deg - 1)) == cudaSuccess ? 0 : -1;
}

int launch_step3(int deg, const Mesh3& m, const Work3& w, double* Q, const Args3& a, void* stream, int block,
                 void** events, int upto) {
  cudaStream_t st = (cudaStream_t)stream;
  if (deg == 1) return step3_impl<1, 4, 2>(m, w, Q, a, st, block, events, upto);
  if (deg == 2) return step3_impl<2, 10, 3>(m, w, Q, a, st, block, events, upto);
  return -2;
}

int step3_launch_count(int want_diag, int shock_limiter) { return 5 + (shock_limiter ? 1 : 0) + (want_diag ? 1 : 0); }

int launch_project3(int deg, int N, int NPJ, double gamma, const double* jw, const double* jphi, const double* prim,
                    double* Q, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = (N + 127) / 128;
  if (deg == 1) k3_project<4><<<grid, 128, 0, st>>>(N, NPJ, gamma, jw, jphi, prim, Q);
  else if (deg == 2) k3_project<10><<<grid, 128, 0, st>>>(N, NPJ, gamma, jw, jphi, prim, Q);
  else return -2;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lxw
