// lxw_kernels3t.cu -- sm_103a kernels of one LxW-DG step on tetrahedral
// meshes: the unstructured 3D extension (end of Sec. 3.3; the 3D Euler
// equations of Sec. 1.1), in the FP64 and the mixed form of the hexahedral
// kernels.
//
// One thread owns one cell, as in the hexahedral form; state Q[N][5][ML].
// Each cell is the affine image of the reference tetrahedron T0; its
// geometry (the inverse Jacobian, the volume and the four outward normals
// scaled by the face areas) is read per cell from a structure of arrays.
// The interior tables live in constant memory (all threads of a warp read
// the same point); the face tables depend on the order in which a face's
// vertices appear in the cell (6 orders per face) and are read from global
// memory through the read-only cache.  Phases as in the hexahedral form:
//   k3t_moment  Sec. 3.1 moment limiter + max |u| + c -> atomicMax
//   k3t_ck      Sec. 2.2-2.3 CK flux: q_t, q_tt carried as modes through the
//               weighted differentiation tables applied to the contravariant
//               flux G_a = sum_d (d r_a / d x_d) F_d; volume integral; traces
//   k3t_face    Sec. 3.3 Step 3 on four faces and Steps 4-5 (Lambda, 15
//               corners, mu)
//   k3t_update  Step 6
//   k3t_shock   Sec. 4.1 with the four face neighbours
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "lxw_internal3d.h"

namespace lxw {
namespace {

__constant__ Tables3T c_tab3t[2];    // degree 1, degree 2
__constant__ Tables3TF c_tab3tf[2];  // their FP32 copies (the mixed form's CK kernel)

#include "lxw_flux3.cuh"

template <typename T>
__device__ __forceinline__ const Tables3TOf<T>& tab3t(int deg);
template <>
__device__ __forceinline__ const Tables3TOf<double>& tab3t<double>(int deg) { return c_tab3t[deg - 1]; }
template <>
__device__ __forceinline__ const Tables3TOf<float>& tab3t<float>(int deg) { return c_tab3tf[deg - 1]; }

template <typename T>
__device__ __forceinline__ const T* face_tables(const Mesh3T& m);
template <>
__device__ __forceinline__ const double* face_tables<double>(const Mesh3T& m) { return m.fphi; }
template <>
__device__ __forceinline__ const float* face_tables<float>(const Mesh3T& m) { return m.fphif; }

// FP32 basis values at limiter point p (the mixed forms' screens)
template <int ML, int NQ, int NF>
__device__ __forceinline__ void load_phif(const Tables3TF& t, const Mesh3T& m, int code, int p, float ph[ML]) {
  if (p < NQ) {
#pragma unroll
    for (int l = 0; l < ML; ++l) ph[l] = t.phi[p][l];
  } else {
    const int k = (p - NQ) / NF, pe = p - NQ - k * NF;
    const float* f = m.fphif + (size_t)((k * k3tPerms + ((code >> (3 * k)) & 7)) * NF + pe) * ML;
#pragma unroll
    for (int l = 0; l < ML; ++l) ph[l] = __ldg(f + l);
  }
}

__device__ __forceinline__ double step_dt3t(const Work3& w, const Mesh3T& m, const Args3& a) {
  const double s = __longlong_as_double((long long)*w.smax);
  return a.dt_in > 0.0 ? a.dt_in : a.cfl * m.hmin / s;
}

__device__ __forceinline__ double geo(const Mesh3T& m, int e, int i) { return m.geo[(size_t)e * m.N + i]; }

// basis values at limiter point p of a cell: interior points from the
// constant bank, face points from the table of the face's vertex order
template <int ML, int NQ, int NF>
__device__ __forceinline__ void load_phi(const Tables3T& t, const Mesh3T& m, int code, int p, double ph[ML]) {
  if (p < NQ) {
#pragma unroll
    for (int l = 0; l < ML; ++l) ph[l] = t.phi[p][l];
  } else {
    const int k = (p - NQ) / NF, pe = p - NQ - k * NF;
    const double* f = m.fphi + (size_t)((k * k3tPerms + ((code >> (3 * k)) & 7)) * NF + pe) * ML;
#pragma unroll
    for (int l = 0; l < ML; ++l) ph[l] = __ldg(f + l);
  }
}

// momentum mirror in the plane of unit normal nh (a reflective wall)
template <typename T>
__device__ __forceinline__ void mirror3(const T nh[3], T q[5]) {
  const T mn = q[1] * nh[0] + q[2] * nh[1] + q[3] * nh[2];
#pragma unroll
  for (int d = 0; d < 3; ++d) q[1 + d] -= T(2) * mn * nh[d];
}

// an . F[.][v] with sign-symmetric rounding: both cells of a face use
// exactly negated normals and must get exactly negated products
template <typename T>
__device__ __forceinline__ T ndot(const T an[3], const T F[3][5], int v) {
  return rn_fma(an[2], F[2][v], rn_fma(an[1], F[1][v], rn_mul(an[0], F[0][v])));
}

// the area of face k of cell i (stored once per face for both of its cells)
__device__ __forceinline__ double face_area(const Mesh3T& m, int k, int i) { return m.geo[(size_t)(22 + k) * m.N + i]; }

// ------------------------------------------------------------ k3t_reset
__global__ void k3t_reset(Work3 w, int want_diag) {
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

// ------------------------------------------------------------ k3t_moment
// Sec. 3.1 Steps 0-2 (Lemma 1's secant) over the interior and face points,
// then |u| + c of the limited state, block max -> atomicMax.
template <int DEG, int ML, int N1>
__global__ void __launch_bounds__(128) k3t_moment(const Mesh3T m, const Work3 w, double* __restrict__ Q,
                                                  const Args3 a) {
  constexpr int NQ = N1 * N1 * N1, NF = N1 * N1, NPT = NQ + 4 * NF;
  const Tables3T& t = c_tab3t[DEG - 1];
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
    const int code = m.code[i];
    auto load = [&](int p, double ph[ML]) { load_phi<ML, NQ, NF>(t, m, code, p, ph); };
    bool screened = false;
    if (a.ck_fp32 && c[0][0] > 0.0) {   // mixed form: the FP32 screen clears unlimited cells
      const double pb = (a.gamma - 1.0) * (c[4][0] - 0.5 * (c[1][0] * c[1][0] + c[2][0] * c[2][0] + c[3][0] * c[3][0]) / c[0][0]);
      if (pb > 0.0) {
        const Tables3TF& tf = tab3t<float>(DEG);
        float cf[5][ML], S[5], smf;
        screen_state3<ML>(c, tf.phimax, cf, S);
        auto loadf = [&](int p, float ph[ML]) { load_phif<ML, NQ, NF>(tf, m, code, p, ph); };
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

// contravariant flux G_a[v] = sum_d Ji[a][d] F_d[v]
template <typename T>
__device__ __forceinline__ void contra3(const T Ji[9], const T F[3][5], T G[3][5]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int v = 0; v < 5; ++v) G[a][v] = Ji[3 * a] * F[0][v] + Ji[3 * a + 1] * F[1][v] + Ji[3 * a + 2] * F[2][v];
}

// q and F_T = F + dt/2 F_t + dt^2/6 F_tt at a point from the basis values
template <typename T, int ML>
__device__ __forceinline__ void ft_point3t(T g1, T c1, T c2, const T ph[ML], const T c[5][ML], const T Qt[5][ML],
                                           const T Qtt[5][ML], T q[5], T FT[3][5]) {
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
  T F[3][5];
  flux3<T>(s, F);
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

// ------------------------------------------------------------ k3t_ck
// Sec. 2.2-2.3 on one cell: Qt = -(projection of div F^h), Qtt likewise
// with F_t, both through W_a applied to G_a; F_T at the interior points
// feeds the volume integral (1/|K|) Int F_T . grad phi_l = sum_k qw_k G_a
// d_a phi_l, the face points store q and an_k . F_T in the trace array.
// T = double: the FP64 form; T = float: the mixed form's FP32 kernel (state
// and volume update in FP64; the traces are stored in T, and the face
// kernel of the same form reads them in T).
template <typename T, int DEG, int ML, int N1>
__global__ void __launch_bounds__(128) k3t_ck(const Mesh3T m, const Work3 w, double* __restrict__ Q, const Args3 a) {
  constexpr int NQ = N1 * N1 * N1, NF = N1 * N1;
  constexpr bool F64 = sizeof(T) == 8;
  const Tables3TOf<T>& t = tab3t<T>(DEG);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const int N = m.N;
  const T g1 = opaque(T(a.gamma - 1.0));
  const double dtd = step_dt3t(w, m, a);
  const T dt = T(dtd);
  const T c1 = opaque(T(0.5 * dtd)), c2 = opaque(T(dtd * dtd / 6.0));
  T Ji[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) Ji[e] = opaque(T(geo(m, e, i)));
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
    T F[3][5], G[3][5];
    flux3<T>(s, F);
    contra3<T>(Ji, F, G);
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int l = 0; l < ML; ++l)
        Qt[v][l] = fmaT(-G[2][v], t.W[2][k][l], fmaT(-G[1][v], t.W[1][k][l], fmaT(-G[0][v], t.W[0][k][l], Qt[v][l])));
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
    T F1[3][5], G[3][5], du[3], dp;
    flux3_d1<T>(g1, s, qt, F1, du, dp);
    contra3<T>(Ji, F1, G);
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int l = 0; l < ML; ++l)
        Qtt[v][l] = fmaT(-G[2][v], t.W[2][k][l], fmaT(-G[1][v], t.W[1][k][l], fmaT(-G[0][v], t.W[0][k][l], Qtt[v][l])));
  }
  // pass 3a: F_T at the interior points -> volume integral of the higher moments
  T Vv[5][ML];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) Vv[v][l] = T(0);
#pragma unroll 1
  for (int p = 0; p < NQ; ++p) {
    T ph[ML], q[5], FT[3][5], G[3][5];
#pragma unroll
    for (int l = 0; l < ML; ++l) ph[l] = t.phi[p][l];
    ft_point3t<T, ML>(g1, c1, c2, ph, c, Qt, Qtt, q, FT);
    contra3<T>(Ji, FT, G);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const T f0 = t.qw[p] * G[0][v], f1 = t.qw[p] * G[1][v], f2 = t.qw[p] * G[2][v];
#pragma unroll
      for (int l = 1; l < ML; ++l)
        Vv[v][l] = fmaT(f0, t.dref[0][p][l], fmaT(f1, t.dref[1][p][l], fmaT(f2, t.dref[2][p][l], Vv[v][l])));
    }
  }
  // pass 3b: traces at the face points, in the face's canonical point order
  const int code = m.code[i];
  const T* ftab = face_tables<T>(m);
#pragma unroll 1
  for (int k = 0; k < 4; ++k) {
    const T an[3] = {T(geo(m, 10 + 3 * k, i)), T(geo(m, 11 + 3 * k, i)), T(geo(m, 12 + 3 * k, i))};
    const T* fk = ftab + (size_t)((k * k3tPerms + ((code >> (3 * k)) & 7)) * NF) * ML;
#pragma unroll 1
    for (int p = 0; p < NF; ++p) {
      T ph[ML], q[5], FTn[5];
#pragma unroll
      for (int l = 0; l < ML; ++l) ph[l] = __ldg(fk + p * ML + l);
      ftn_point3<T, ML>(g1, c1, c2, an, ph, c, Qt, Qtt, q, FTn);   // an . F_T directly
      T* tr = reinterpret_cast<T*>(w.trace) + ((size_t)(k * NF + p) * 10) * N + i;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        tr[(size_t)v * N] = q[v];
        tr[(size_t)(5 + v) * N] = FTn[v];
      }
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

// ------------------------------------------------------------ k3t_face
// Sec. 3.3 Step 3 on the four faces, seen from each cell: both cells of a
// face take its points in the same order, exactly negated normals and the
// same sign-symmetric rounded operations, so their LLF values, f^LxW and
// f^LxF are exact negatives.  Face integral of the higher moments; Steps
// 4-5: Gamma, the density Lambda shared by the negative faces, the
// Lax-Friedrichs state, mu over the 15 corners of the box of proposals.
// T is the arithmetic of the point loop (FP32 in the mixed form); the
// averages, f^LxF and Steps 4-5 are FP64 in both forms.
template <typename T, int DEG, int ML, int N1>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1) k3t_face(const Mesh3T m, const Work3 w, double* __restrict__ Q,
                                                const Args3 a) {
  constexpr int NF = N1 * N1;
  const Tables3TOf<T>& t = tab3t<T>(DEG);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const int N = m.N;
  const double g = a.gamma, g1 = g - 1.0;
  const T gT = T(g);
  const double s = __longlong_as_double((long long)*w.smax);
  const double dt = step_dt3t(w, m, a);
  const double vol = geo(m, 9, i);
  const int code = m.code[i];
  const T* trb = reinterpret_cast<const T*>(w.trace);
  const T* ftab = face_tables<T>(m);
  double* Qi = Q + (size_t)i * 5 * ML;
  double qb[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) qb[v] = Qi[v * ML];
  double Fb[3][5];   // the average's flux, from the moment kernel
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int v = 0; v < 5; ++v) Fb[d][v] = w.fbar[(size_t)(d * 5 + v) * N + i];
  T Ei[5][ML];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int l = 0; l < ML; ++l) Ei[v][l] = T(0);
  double fW[4][5], fF[4][5];
#pragma unroll 1
  for (int k = 0; k < 4; ++k) {
    const int j = m.nbr[k * N + i], kj = (code >> (12 + 2 * k)) & 3;
    const double an[3] = {geo(m, 10 + 3 * k, i), geo(m, 11 + 3 * k, i), geo(m, 12 + 3 * k, i)};
    const double area = face_area(m, k, i);
    const bool wall = j < 0 && -1 - j == LXW_BC_REFLECT;
    double nh[3] = {0.0, 0.0, 0.0};   // the unit normal, needed on walls only
    if (wall) { nh[0] = an[0] / area; nh[1] = an[1] / area; nh[2] = an[2] / area; }
    const double hs = 0.5 * s * area;
    double qn[5];
    if (j >= 0) {
      const double* Qj = Q + (size_t)j * 5 * ML;
#pragma unroll
      for (int v = 0; v < 5; ++v) qn[v] = Qj[v * ML];
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) qn[v] = qb[v];
      if (wall) mirror3<double>(nh, qn);
    }
    {
      // a neighbour's average flux from the moment kernel, a wall's mirrored state here
      double Fn[3][5];
      if (j >= 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int v = 0; v < 5; ++v) Fn[d][v] = w.fbar[(size_t)(d * 5 + v) * N + j];
      } else if (wall) {
        const P3 sn = make_p3(g1, qn);
        flux3(sn, Fn);
      } else {
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int v = 0; v < 5; ++v) Fn[d][v] = Fb[d][v];
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double ai = ndot<double>(an, Fb, v), ak = ndot<double>(an, Fn, v);
        fF[k][v] = __fma_rn(-hs, __dsub_rn(qn[v], qb[v]), __dmul_rn(0.5, __dadd_rn(ai, ak)));
      }
    }
    T fWk[5] = {T(0), T(0), T(0), T(0), T(0)};
    const T hsT = T(hs), sT = T(s), areaT = T(area);
    const T nhT[3] = {T(nh[0]), T(nh[1]), T(nh[2])};
    const T* fk = ftab + (size_t)((k * k3tPerms + ((code >> (3 * k)) & 7)) * NF) * ML;
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
      } else if (wall) {
        // exterior R q, and n . F_T(R q) = -R (n . F_T(q)) (the Euler flux's mirror symmetry)
#pragma unroll
        for (int v = 0; v < 5; ++v) { qx[v] = qi[v]; Fx[v] = Fi[v]; }
        mirror3<T>(nhT, qx);
        mirror3<T>(nhT, Fx);
#pragma unroll
        for (int v = 0; v < 5; ++v) Fx[v] = -Fx[v];
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) { qx[v] = qi[v]; Fx[v] = Fi[v]; }
      }
      const T hp = a.llf_global ? hsT : T(0.5) * fminT(sT, fmaxT(lf_speed3<T>(gT, qi), lf_speed3<T>(gT, qx))) * areaT;
      T ph[ML];
#pragma unroll
      for (int l = 1; l < ML; ++l) ph[l] = __ldg(fk + p * ML + l);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const T fs = rn_fma(-hp, rn_sub(qx[v], qi[v]), rn_mul(T(0.5), rn_add(Fi[v], Fx[v])));
        fWk[v] = rn_fma(t.fw[p], fs, fWk[v]);
        const T hw = t.fw[p] * fs;
#pragma unroll
        for (int l = 1; l < ML; ++l) Ei[v][l] = fmaT(hw, ph[l], Ei[v][l]);
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) fW[k][v] = double(fWk[v]);
  }
  const double dta = dt / vol;
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int l = 1; l < ML; ++l) Qi[v * ML + l] -= dta * double(Ei[v][l]);

  // Steps 4-5
  double Gam0 = vol / dt * qb[0];
#pragma unroll
  for (int k = 0; k < 4; ++k) Gam0 -= fF[k][0];
  if (Gam0 < 0.0) atomicOr(w.status, (unsigned)LXW_ST_CFL);
  double neg = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double df = fF[k][0] - fW[k][0];
    if (df < 0.0) neg += df;
  }
  double ql[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) acc += fF[k][v];
    ql[v] = qb[v] - dta * acc;
  }
  const double er = fmax(fmin(a.eps0, 0.5 * ql[0]), 0.0);
  double lneg = 1.0;
  if (neg < 0.0) lneg = fmin(1.0, fmax(0.0, (Gam0 - vol / dt * er) / (-neg)));
  double lam[4], dq[4][5];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    lam[k] = (fF[k][0] - fW[k][0]) < 0.0 ? lneg : 1.0;
#pragma unroll
    for (int v = 0; v < 5; ++v) dq[k][v] = dta * lam[k] * (fF[k][v] - fW[k][v]);
  }
  const double pl =
      ql[0] > 0.0 ? g1 * (ql[4] - 0.5 * (ql[1] * ql[1] + ql[2] * ql[2] + ql[3] * ql[3]) / ql[0]) : -1.0;
  double mmin[4] = {1.0, 1.0, 1.0, 1.0};
  if (!(ql[0] > 0.0) || !(pl > 0.0)) {
#pragma unroll
    for (int k = 0; k < 4; ++k) mmin[k] = 0.0;
  } else {
    const double kap = fmin(a.eps0, 0.5 * pl) / g1;
    const double h0 = ql[0] * ql[4] - 0.5 * (ql[1] * ql[1] + ql[2] * ql[2] + ql[3] * ql[3]) - kap * ql[0];
    // every corner ql + dd has |dd_v| <= D_v = sum_k |dq_kv|, so h(ql + dd) >= h0
    // - (|rho| D_E + |E - kappa| D_rho + |m| . D_m) - (D_rho D_E + |D_m|^2 / 2):
    // when that bound (and rho - D_rho) clears zero by more than the rounding,
    // every corner is positive and every mu is 1 without the corner loop
    double D[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int v = 0; v < 5; ++v) D[v] += fabs(dq[k][v]);
    const double lin = fabs(ql[0]) * D[4] + fabs(ql[4] - kap) * D[0] + fabs(ql[1]) * D[1] + fabs(ql[2]) * D[2] +
                       fabs(ql[3]) * D[3];
    const double quad = D[0] * D[4] + 0.5 * (D[1] * D[1] + D[2] * D[2] + D[3] * D[3]);
    const double scale = fabs(ql[0] * ql[4]) + 0.5 * (ql[1] * ql[1] + ql[2] * ql[2] + ql[3] * ql[3]) +
                         fabs(kap * ql[0]) + lin + quad;
    const bool all_pos = ql[0] - D[0] > 1e-12 * ql[0] && h0 - lin - quad > 1e-12 * scale;
#pragma unroll 1
    for (int cm = all_pos ? 16 : 1; cm < 16; ++cm) {
      double dd[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 0; k < 4; ++k)
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
      for (int k = 0; k < 4; ++k)
        if ((cm >> k) & 1) mmin[k] = fmin(mmin[k], mu);
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    w.prop[k * N + i] = lam[k] * mmin[k];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      w.flux[(size_t)(k * 10 + v) * N + i] = fW[k][v];
      w.flux[(size_t)(k * 10 + 5 + v) * N + i] = fF[k][v];
    }
  }
}

// ------------------------------------------------------------ k3t_update
// Sec. 3.3 Step 6: theta of a face = min of the two cells' proposals;
// blended update of the averages.
template <int ML>
__global__ void __launch_bounds__(128) k3t_update(const Mesh3T m, const Work3 w, double* __restrict__ Q,
                                                  const Args3 a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const int N = m.N;
  const double dt = step_dt3t(w, m, a);
  const int code = m.code[i];
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int j = m.nbr[k * N + i], kj = (code >> (12 + 2 * k)) & 3;
    double th = w.prop[k * N + i];
    if (j >= 0) th = fmin(th, w.prop[kj * N + j]);
    if (a.theta_face) a.theta_face[(size_t)i * 4 + k] = th;
    // count each face once: from the lower cell (lower local face when a
    // cell meets itself across a period), or from the cell of a boundary face
    if (a.want_diag && th < 1.0 && (j < 0 || i < j || (i == j && k < kj))) atomicAdd(&w.diag->nface, 1ull);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double fw = w.flux[(size_t)(k * 10 + v) * N + i], ff = w.flux[(size_t)(k * 10 + 5 + v) * N + i];
      acc[v] += th * fw + (1.0 - th) * ff;
    }
  }
  double* Qi = Q + (size_t)i * 5 * ML;
  const double dta = dt / geo(m, 9, i);
#pragma unroll
  for (int v = 0; v < 5; ++v) Qi[v * ML] -= dta * acc[v];
}

// ------------------------------------------------------------ k3t_shock
// Sec. 4.1 on (rho, u, v, w, p) with the four face neighbours (a wall's
// exterior: the mirrored average), alpha = alpha0 dx^1.5 with dx = |K|^(1/3).
template <int DEG, int ML, int N1>
__global__ void __launch_bounds__(128) k3t_shock(const Mesh3T m, const Work3 w, double* __restrict__ Q,
                                                 const Args3 a) {
  constexpr int NQ = N1 * N1 * N1, NF = N1 * N1, NPT = NQ + 4 * NF;
  const Tables3T& t = c_tab3t[DEG - 1];
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
    const int code = m.code[i];
    if (a.ck_fp32) {   // mixed form: FP32 bounds and points clear cells well inside [m, M]
      const Tables3TF& tf = tab3t<float>(DEG);
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
          if (-1 - j == LXW_BC_REFLECT) {
            const double an[3] = {geo(m, 10 + 3 * k, i), geo(m, 11 + 3 * k, i), geo(m, 12 + 3 * k, i)};
            const double area = face_area(m, k, i);
            const float nh[3] = {(float)(an[0] / area), (float)(an[1] / area), (float)(an[2] / area)};
            mirror3<float>(nh, qn);
          }
        }
        return true;
      };
      auto loadf = [&](int p, float ph[ML]) { load_phif<ML, NQ, NF>(tf, m, code, p, ph); };
      const float alf = (float)a.alpha0 * powf(cbrtf((float)geo(m, 9, i)), 1.5f);
      if (shock_bounds3<4>((float)a.gamma, alf, qbf, nbrf, hi, lo) &&
          shock_screen3<ML, NPT>(cf, S, (float)a.gamma, hi, lo, loadf))
        return;
    }
    double qb[5], wb[5], Mx[5], Mn[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qb[v] = c[v][0];
    prim(qb, wb);
    const double al = a.alpha0 * pow(cbrt(geo(m, 9, i)), 1.5);
#pragma unroll
    for (int v = 0; v < 5; ++v) { Mx[v] = wb[v] + al; Mn[v] = wb[v] - al; }
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
      const int j = m.nbr[k * N + i];
      double qn[5], wn[5];
      if (j >= 0) {
        const double* Qj = Q + (size_t)j * 5 * ML;
#pragma unroll
        for (int v = 0; v < 5; ++v) qn[v] = Qj[v * ML];
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) qn[v] = qb[v];
        if (-1 - j == LXW_BC_REFLECT) {
          const double an[3] = {geo(m, 10 + 3 * k, i), geo(m, 11 + 3 * k, i), geo(m, 12 + 3 * k, i)};
          const double area = face_area(m, k, i);
          const double nh[3] = {an[0] / area, an[1] / area, an[2] / area};
          mirror3<double>(nh, qn);
        }
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
      double ph[ML], q[5], wp[5];
      load_phi<ML, NQ, NF>(t, m, code, p, ph);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double acc = 0.0;
#pragma unroll
        for (int l = 0; l < ML; ++l) acc = fma(c[v][l], ph[l], acc);
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

// ------------------------------------------------------------ k3t_diag
// Totals |K| Q^(1) and minimum density / pressure of the averages.
template <int ML>
__global__ void __launch_bounds__(256) k3t_diag(const Mesh3T m, const Work3 w, const double* __restrict__ Q,
                                                double gamma) {
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
    const double vol = geo(m, 9, i);
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] *= vol;
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

template <int DEG, int ML, int N1>
int step3t_impl(const Mesh3T& m, const Work3& w, double* Q, const Args3& a, cudaStream_t st, int block, void** events,
                int upto) {
  const int grid = (m.N + block - 1) / block;
  int ne = 0;
  auto mark = [&]() { if (events) cudaEventRecord((cudaEvent_t)events[ne++], st); };
  auto ok = [&]() { return cudaGetLastError() == cudaSuccess ? 0 : -1; };
  k3t_reset<<<1, 32, 0, st>>>(w, a.want_diag);
  mark();
  k3t_moment<DEG, ML, N1><<<grid, block, 0, st>>>(m, w, Q, a);
  mark();
  if (upto < 2) return ok();
  if (a.ck_fp32) k3t_ck<float, DEG, ML, N1><<<grid, block, 0, st>>>(m, w, Q, a);
  else k3t_ck<double, DEG, ML, N1><<<grid, block, 0, st>>>(m, w, Q, a);
  mark();
  if (upto < 3) return ok();
  if (a.ck_fp32) k3t_face<float, DEG, ML, N1><<<grid, block, 0, st>>>(m, w, Q, a);
  else k3t_face<double, DEG, ML, N1><<<grid, block, 0, st>>>(m, w, Q, a);
  mark();
  if (upto < 4) return ok();
  k3t_update<ML><<<grid, block, 0, st>>>(m, w, Q, a);
  mark();
  if (upto < 5) return ok();
  if (a.shock_limiter) k3t_shock<DEG, ML, N1><<<grid, block, 0, st>>>(m, w, Q, a);
  mark();
  if (a.want_diag) k3t_diag<ML><<<(m.N + 255) / 256, 256, 0, st>>>(m, w, Q, a.gamma);
  return ok();
}

}  // namespace

int upload_tables3t(int deg, const Tables3T& t) {
  if (deg < 1 || deg > 2) return -1;
  Tables3TF f;
  const double* src = &t.qw[0];
  float* dst = &f.qw[0];
  static_assert(sizeof(Tables3T) == 2 * sizeof(Tables3TF), "tables hold doubles only");
  for (size_t k = 0; k < sizeof(Tables3T) / sizeof(double); ++k) dst[k] = (float)src[k];
  if (cudaMemcpyToSymbol(c_tab3t, &t, sizeof(Tables3T), sizeof(Tables3T) * (deg - 1)) != cudaSuccess) return -1;
  return cudaMemcpyToSymbol(c_tab3tf, &f, sizeof(Tables3TF), sizeof(Tables3TF) * (deg - 1)) == cudaSuccess ? 0 : -1;
}

int launch_step3t(int deg, const Mesh3T& m, const Work3& w, double* Q, const Args3& a, void* stream, int block,
                  void** events, int upto) {
  cudaStream_t st = (cudaStream_t)stream;
  if (deg == 1) return step3t_impl<1, 4, 2>(m, w, Q, a, st, block, events, upto);
  if (deg == 2) return step3t_impl<2, 10, 3>(m, w, Q, a, st, block, events, upto);
  return -2;
}

}  // namespace lxw
