// lxw_internal3d.h -- shared declarations of the 3D FP64 forms on hexahedra
// (Cartesian boxes) and tetrahedra: tables, device views, launchers.  Not
// part of the public ABI.
#pragma once

#include "lxw_internal.h"

namespace lxw {

// Degrees 1 and 2: at most 10 modes, 3 Gauss points per direction.
constexpr int k3MaxML = 10;
constexpr int k3MaxN = 3;
constexpr int k3MaxQ = k3MaxN * k3MaxN * k3MaxN;   // interior points
constexpr int k3MaxF = k3MaxN * k3MaxN;            // points per face
constexpr int k3MaxPts = k3MaxQ + 6 * k3MaxF;      // limiter points: interior, then faces
constexpr int k3MaxProj = 125;                     // projection points ((deg + 3)^3)

// Reference-cube tables of one degree.  Points: the interior tensor Gauss
// points (xi fastest), then face k's points at NQ + k NF + t n + u, with u
// along the first and t along the second tangential axis (x, y, z order),
// so that the two cells of a face meet its points in the same order.
template <typename T>
struct Tables3Of {
  T qw[k3MaxQ];                        // interior weights, sum 1
  T fw[k3MaxF];                        // face weights, sum 1
  T phi[k3MaxPts][k3MaxML];            // basis at every point
  T dref[3][k3MaxQ][k3MaxML];          // d phi / d(xi, eta, zeta) at the interior points
  T W[3][k3MaxQ][k3MaxML];             // qw_k sum_m phi_m(x_k) D_d[m][l], D_d[m][l] = (1/8) Int d_d phi_m phi_l
  T phimax[k3MaxML];                   // max over the limiter points of |phi_l| (the FP32 screens' bound)
};
using Tables3 = Tables3Of<double>;     // FP64 forms
using Tables3F = Tables3Of<float>;     // the FP32 CK kernel of the mixed forms

// Uniform box cells: one spacing per axis.
struct Mesh3 {
  int N, nx, ny, nz;
  double h[3], vol, hmin;              // hmin = 3 |K| / |dK|
  const int* nbr;                      // [6][N]: neighbour across face k, or -1 - bc
};

struct Diag3Block {
  double sum[5];
  unsigned long long minr, minp;       // order-preserving bits of min rho, min p
  unsigned long long nmom, nface, nsc;
};

struct Work3 {
  double* trace;                       // [E][NF][10][N]: q (5), n_out . F_T (5), n scaled by the face area
  double* flux;                        // [E][10][N]: outward f^LxW (5), f^LxF (5)
  double* prop;                        // [E][N]: flux-limiter proposals
  double* fbar;                        // [3][5][N]: Euler flux of each cell's average (moment kernel)
  unsigned long long* smax;            // bits of the global wave speed (non-negative double)
  unsigned int* status;                // LXW_ST_* bits of the step
  Diag3Block* diag;
};

struct Args3 {
  double dt_in, cfl, gamma, eps0, alpha0;
  int shock_limiter, llf_global, want_diag;
  int ck_fp32;                         // mixed form: FP32 CK and face point loops, FP32 screens in the
                                       // moment and shock limiters (state, decisions in FP64)
  double* theta_face;                  // [N][E] or null
};

// Tables of one degree into the device's constant bank, with their FP32
// copy (synchronous).
int upload_tables3(int deg, const Tables3& t);
// One step: reset, moment, ck, face, update, shock (if on), diag (if asked).
// events (nullable): recorded before each phase and after the last; upto:
// phases to run (1 moment .. 5 shock).
int launch_step3(int deg, const Mesh3& m, const Work3& w, double* Q, const Args3& a, void* stream, int block,
                 void** events, int upto);
int step3_launch_count(int want_diag, int shock_limiter);
// Q[N][5][ML] = L2 projection of prim[N][NPJ][5] = (rho, u, v, w, p) with the
// projection weights jw[NPJ] and basis jphi[NPJ][ML] (device arrays).
int launch_project3(int deg, int N, int NPJ, double gamma, const double* jw, const double* jphi, const double* prim,
                    double* Q, void* stream);

// ---------------------------------------------------------------- tetrahedra
// Reference cell T0 = {r, s, t >= 0, r + s + t <= 1}, affine map from the
// cell's vertices 0..3.  Interior points: a conical product of Gauss-Jacobi
// rules, (deg + 1)^3 points; face k (opposite vertex k): a collapsed
// triangle rule with (deg + 1)^2 points placed from the face's vertices in
// ascending vertex-id order, so both cells of a face meet its points in one
// order.  Face k's vertices appear in one of 6 orders ("perm").
constexpr int k3tPerms = 6;

template <typename T>
struct Tables3TOf {
  T qw[k3MaxQ];                        // interior weights, sum 1
  T fw[k3MaxF];                        // face weights, sum 1
  T phi[k3MaxQ][k3MaxML];              // basis at the interior points
  T dref[3][k3MaxQ][k3MaxML];          // d phi / d(r, s, t) there
  T W[3][k3MaxQ][k3MaxML];             // qw_k sum_m phi_m(x_k) D_a[m][l], D_a[m][l] = (1/|T0|) Int d_a phi_m phi_l
  T phimax[k3MaxML];                   // max over the interior and every face table of |phi_l|
};
using Tables3T = Tables3TOf<double>;
using Tables3TF = Tables3TOf<float>;

// Per-cell geometry, structure of arrays.
constexpr int k3tGeo = 26;             // Ji (9), vol, an (4 x 3), face areas (4)
struct Mesh3T {
  int N;
  double hmin;                         // min 3 |K| / |dK|
  const double* geo;                   // [26][N]: Ji[a][d] = d r_a / d x_d (row-major), |K|, outward
                                       //   normals scaled by the face area (face k: 10 + 3k ..), the
                                       //   face areas (face k: 22 + k; one value for both cells)
  const int* nbr;                      // [4][N]: neighbour across face k, or -1 - bc
  const int* code;                     // [N]: bits 3k..3k+2 perm of face k, bits 12+2k..12+2k+1 the
                                       //   neighbour's local face
  const double* fphi;                  // [4][6][NF][ML]: basis at the face points (device, read-only)
  const float* fphif;                  // the same in FP32 (mixed forms)
};

int upload_tables3t(int deg, const Tables3T& t);
int launch_step3t(int deg, const Mesh3T& m, const Work3& w, double* Q, const Args3& a, void* stream, int block,
                  void** events, int upto);

// Host quadrature helpers shared with the 2D tables (lxw_host.cpp).
void host_gauss_legendre(int n, double* x, double* w);
void host_legendre_norm(int n, double x, double& v, double& d);

}  // namespace lxw
