// lxw_internal.h -- data structures shared by the library's host code
// (lxw_host.cpp) and its CUDA kernels (lxw_kernels.cu).
#pragma once
#include <cstddef>
#include <cstdint>

#include "../../include/lxw.h"

namespace lxw {

constexpr int kMaxML = 10;
constexpr int kMaxQ = 16;     // interior points (degree 3: 4 x 4)
constexpr int kMaxMQ = 4;     // points per edge
constexpr int kMaxE = 4;
constexpr int kMaxPts = kMaxQ + kMaxE * kMaxMQ;
constexpr int kMaxProj = 36;  // (degree + 3)^2 projection points

// Quadrature and basis tables of one (element kind, degree).  Kept in the
// device's __constant__ bank: every thread of a warp reads the same entry at
// the same time, so the accesses are broadcasts.
struct Tables {
  int ML, NQ, MQ, E, NPT, NPJ;
  double w[kMaxQ];                 // interior weights, sum 1
  double ew[kMaxMQ];               // edge Gauss-Legendre weights, sum 2
  double phi[kMaxPts][kMaxML];     // basis at interior points then edge points
  double dxi[kMaxPts][kMaxML];     // d phi / d xi
  double deta[kMaxPts][kMaxML];    // d phi / d eta
};

// Projection tables (initial condition only).
struct ProjTables {
  int ML, NPJ;
  double w[kMaxProj];
  double phi[kMaxProj][kMaxML];
};

// Device geometry, structure of arrays indexed [.. ][N] so that one thread
// per element reads coalesced.
struct DevMesh {
  int N, E;
  const double* area;     // [N]
  const double* jinv;     // [4][N]: dxi/dx, dxi/dy, deta/dx, deta/dy
  const double* nrm;      // [E][2][N]: outward normal scaled by edge length
  const double* sdx;      // [N]: spacing for the shock limiter alpha
  const int* nbr;         // [E][N]: neighbour id, or -1 - bc code on the boundary
  const int* nbk;         // [E][N]: neighbour's local edge
  double hmin;            // min_i 2|T_i| / P_i
  // FP32 copies for the mixed form (null for FP64 solvers)
  const float* jinv32;    // [4][N]
  const float* nrm32;     // [E][2][N]
  const float* sdx32;     // [N]
  const float* inva32;    // [N]: 1 / |T_i|
  const double* inva;     // [N]: 1 / |T_i|
  // mixed form work list: tiles (start element, count, problem id, 0); each
  // problem is a contiguous element range, hmin per problem
  const int4* tiles;
  int ntiles;
  int nprob;
  const double* hmin_p;   // [nprob]
};

// Device workspace of one solver.
struct DevWork {
  double* trace;          // [E][MQ][8][N]: q (4) and n_out . F_T (4) at edge points
  double* flux;           // [E][8][N]: outward f^LxW (4), f^LxF (4)
  double* prop;           // [E][N]: Lambda proposals
  unsigned long long* smax;  // wave speed (bits of a non-negative double)
  unsigned int* status;      // LXW_ST_* bits
  double* diag;           // [16] reduction slots (see lxw_kernels.cu)
};

// Per-step scalars of the mixed form, computed once on the device.
struct ScalMx {
  double s, dt;           // wave speed (inflated FP32 maximum) and time step
  float s32, dt32, c1, c2;  // FP32: s, dt, dt/2, dt^2/6
  int live;               // 0: the problem has reached the end time of a timed run (its kernels skip it)
};

// Workspace of the mixed-precision form (FP32 bulk, FP64 averages).
struct DevWorkMx {
  float* trace;           // [E][MQ][8][N]: q (4) and n_out . F_T (4), FP32
  float* fw;              // [E][4][N]: outward f^LxW, FP32 sums
  float* prop;            // [E][N]: Lambda proposals, rounded down to FP32
  double* avg_new;        // [4][N]: updated averages before the shock limiter commits them
  float* avgn32;          // [4][N]: FP32 copy of avg_new
  ScalMx* scal;           // [nprob]
  unsigned long long* smax;  // [nprob]
  unsigned int* status;
  double* diag;           // DiagBlock
  unsigned int* done;     // CTAs of the moment kernel that have finished (the last one computes scal)
  int* gate_list;         // [N]: cells the shock limiter's exact screen left, for the gated limiter
  unsigned int* gate_count;  // entries of gate_list (zeroed by the update kernel every step)
};

// Diagnostics block on the device (both forms).
struct DiagBlock {
  double sum[4];
  unsigned long long minr, minp;      // order-preserving bits of min rho, min p
  unsigned long long nmom, nedge, nsc;
  unsigned long long fb_mom, fb_edge; // mixed form: cells that took the FP64 limiter path
  unsigned long long mlp_skip;        // cells whose shock-limiter work the learned gate skipped
};

// Learned troubled-cell indicator: MLP 24 -> 64 (ReLU) -> 64 (ReLU) -> 1
// (sigmoid).  Parameter vector (float): W1[24][64], b1[64], W2[64][64],
// b2[64], w3[64], b3.
constexpr int kMlpIn = 24, kMlpH = 64;
constexpr int kW1 = 0, kB1 = kW1 + kMlpIn * kMlpH, kW2 = kB1 + kMlpH, kB2 = kW2 + kMlpH * kMlpH,
              kW3 = kB2 + kMlpH, kB3 = kW3 + kMlpH, kMlpParams = kB3 + 1;

// The gate's weights as the shared-memory image the gate kernel's tensor-core
// products read: W1^T [64 x 32] (24 inputs, zero padded) and W2^T [64 x 64]
// in BF16, each in the K-major, unswizzled core-matrix layout of tcgen05
// operands (8 rows x 16 bytes per core matrix, core matrices along K 128 B
// apart, 8-row groups K/8 x 128 B apart); biases, output weights and output
// bias are the BF16 values widened to FP32; then the per-feature bounds
// inside which the network's prediction is used.
constexpr int kGateK1 = 32;
__host__ __device__ constexpr int umma_kmajor(int r, int k, int K) {
  return (((r >> 3) * (K >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}
struct GateWeights {
  unsigned short w1[kMlpH * kGateK1];
  unsigned short w2[kMlpH * kMlpH];
  float b1[kMlpH], b2[kMlpH], w3[kMlpH], b3, pad[3];
  float lo[kMlpIn], hi[kMlpIn];      // envelope of the training features (the gate skips only inside it)
};
static_assert(sizeof(GateWeights) % 16 == 0, "GateWeights is copied in 16-byte words");

struct StepArgs {
  int grid;                          // mixed form: persistent CTAs (0 = one per tile)
  double dt_in, cfl, gamma, eps0, alpha0;
  float gamma_f, eps0_f, alpha0_f;   // FP32 copies for the mixed form
  int sms;                           // SMs of the device
  int gate_per_sm;                   // resident CTAs per SM of the gated shock kernel (its persistent grid)
  int hi_occupancy;                  // mixed form: the edge / gated-shock variants with more CTAs per SM
  const GateWeights* gate_w;         // learned gate weights or null
  float mlp_tau;                     // gate: skip the limiter where theta_hat >= 1 - tau
  long long gate_wait_test;          // > 0: each gate CTA first waits this many cycles on a barrier nothing arrives at (test aid)
  float* feat_out;                   // [N][24] features at the shock limiter's input, or null
  float* gate_out;                   // [N] network output theta_hat (needs the gate), or null
  double qin[4];                     // conserved state of LXW_BC_INFLOW faces
  double fin[4], gin[4];             // its Euler fluxes F(q_in), G(q_in)
  float qin32[4], fin32[4], gin32[4];  // FP32 copies (mixed form)
  int shock_limiter;
  int moment_exact;                  // moment limiter: exact root instead of the secant
  int llf_global;                    // LLF point flux: global s instead of the local speed of the traces
  int ck_order;                      // CK flux order in time: 3 (Eq. taylor3-flux) or 4
  int gate_scan;                     // gated limiter: 1 = the gate kernel screens every cell, 0 = list
  int want_diag;
  double* theta_cell;     // [2][N] or null
  double* theta_edge;     // [N][E] or null
  // timed runs (lxw_run_to): each problem steps until its clock reaches
  // t_end, the last step shortened to land on it; tclock[4 p + (0..3)] =
  // elapsed time, steps taken, dt and s of the last step taken
  int timed;
  double t_end;
  double* tclock;
};

// Kernel launchers (lxw_kernels.cu).  All enqueue on `stream`, allocate nothing.
// Writes an MLP's parameters, rounded to BF16, into a device GateWeights
// (lxw_mlp.cu); synchronises the MLP's stream.  0 on success.
int mlp_gate_weights(lxw_mlp* n, GateWeights* out_dev);
// Sets the message lxw_last_error() returns on this thread.
void set_last_error(const char* msg);
// Builds the quadrature / basis tables of one (kind, degree) on the host.
void make_tables(int kind, int deg, Tables& t);
// Copies the tables of one (kind, degree) into the device's constant bank
// (synchronous; done when a solver is created on the current device).
int upload_tables(int kind, int deg, const Tables& t);
// events (nullable): ev[0..launches] recorded before each launch and after the last
// upto: number of phases to run (1 moment .. 5 shock; larger = all)
int launch_step(int kind, int deg, const DevMesh& m, const DevWork& w,
                double* Q, const StepArgs& a, void* stream, int block, void** events = nullptr,
                int upto = 99);
int launch_moment_limit(int kind, int deg, const DevMesh& m, const DevWork& w,
                        double* Q, const StepArgs& a, double* theta, void* stream, int block);
int launch_shock_limit(int kind, int deg, const DevMesh& m, double* Q,
                       const StepArgs& a, double* theta, void* stream, int block);
int launch_project(const ProjTables& t, int N, double gamma, const double* prim, double* Q,
                   void* stream);
int launch_copy_speed(const DevWork& w, double* s_dev, void* stream);
int step_launch_count(int want_diag, int shock_limiter);

// Mixed-precision form (lxw_kernels_mx.cu).  State layout: averages double
// [4][N], an FP32 copy of the averages float [4][N], higher modes float
// [4][ML-1][N].
// Weighted differentiation tables: W[d][k][l] = w_k sum_m phi_m(x_k) D_d[m][l]
// with D_d[m][l] = (1/|T0|) Int d(phi_m)/d(xi_d) phi_l (exact by the interior
// rule), so that the modal coefficients of div F^h are
// -sum_k (W[0][k][l] F_xi(x_k) + W[1][k][l] F_eta(x_k)).
struct DerivTables {
  double W[2][kMaxQ][kMaxML];
};
void make_deriv_tables(const Tables& t, DerivTables& d);
int upload_tables_mx(int kind, int deg, const Tables& t);
// resident CTAs per SM of the gate kernel for (kind, deg), capped by TMEM; < 0 on error
int gate_occupancy(int kind, int deg, int hi_occupancy);
int launch_step_mx(int kind, int deg, const DevMesh& m, const DevWorkMx& w, double* state,
                   const StepArgs& a, void* stream, int block, void** events = nullptr, int upto = 99);
int launch_moment_limit_mx(int kind, int deg, const DevMesh& m, const DevWorkMx& w, double* state,
                           const StepArgs& a, double* theta, void* stream, int block);
int launch_pack(int ML, int N, const double* Q64, double* state, void* stream);
int launch_unpack(int ML, int N, const double* state, double* Q64, void* stream);

}  // namespace lxw
