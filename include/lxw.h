/*
 * lxw.h -- C ABI of the GB300 (sm_103a) library for one time step of the
 * positivity-preserving Lax-Wendroff discontinuous Galerkin (LxW-DG) method
 * for the 2D compressible Euler equations (Moe, Rossmanith & Seal,
 * arXiv:1601.08145), on axis-aligned Cartesian and unstructured triangle
 * meshes, polynomial degree 2 or 3.
 *
 * Every call returns lxw_status (LXW_OK = 0); no C++ exception crosses the
 * boundary.  On failure lxw_last_error() returns a thread-local message.
 * Pointers named *_dev are CUDA device pointers owned by the caller; *_host
 * pointers are host memory owned by the caller.  Meshes and solvers are
 * opaque, owned by the library and released by their destroy calls.
 *
 * State layout (Sec. 1.2, modal expansion q^h = sum_l Q^(l) phi^(l)):
 *   Q[N][4][ML] doubles, element-major; variables (rho, rho u, rho v, E);
 *   mode l = 0 is the cell average (phi^(1) = 1).  ML = 6 (P2) or 10 (P3).
 *   Quadrilateral modes (reference square [-1,1]^2, normalised Legendre
 *   L_n with (1/2) Int L_n^2 = 1): 1, L1(x), L1(y), L1(x)L1(y), L2(x),
 *   L2(y) [, L3(x), L2(x)L1(y), L1(x)L2(y), L3(y)].  Triangle modes
 *   (reference {x,y >= 0, x+y <= 1}): Gram-Schmidt of 1, x, y, x^2, xy,
 *   y^2 [, x^3, x^2y, xy^2, y^3] under (1/|T0|) Int, positive leading term.
 *
 * Boundary codes: LXW_BC_PERIODIC (Cartesian, paired sides),
 * LXW_BC_REFLECT (solid wall) and LXW_BC_TRANSPARENT (outflow), Sec. 2.4;
 * LXW_BC_INFLOW (a steady prescribed state, lxw_solver_set_inflow), the
 * inflow side of the shock-diffraction problem of Sec. 4.
 */
#ifndef LXW_H
#define LXW_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LXW_OK = 0,
  LXW_ERR_ARG = 1,          /* invalid argument (message says which)              */
  LXW_ERR_CUDA = 2,         /* a CUDA runtime call failed                          */
  LXW_ERR_NONPOSITIVE = 3,  /* an input cell average had rho <= 0 or p <= 0        */
  LXW_ERR_CFL = 4,          /* Gamma^rho < 0: dt above the low-order CFL bound      */
  LXW_ERR_NAN = 5,          /* a non-finite value appeared in the state            */
  LXW_ERR_BOUNDS = 6,       /* mesh connectivity out of range                      */
  LXW_ERR_TIMEOUT = 7,      /* a bounded device wait (tensor-core gate) gave up    */
  LXW_ERR_NOMEM = 8         /* device or host allocation failed                    */
} lxw_status;

enum { LXW_BC_PERIODIC = 0, LXW_BC_REFLECT = 1, LXW_BC_TRANSPARENT = 2, LXW_BC_INFLOW = 3 };
enum { LXW_KIND_QUAD = 0, LXW_KIND_TRI = 1 };
/* Precision forms.  LXW_PREC_FP64: every operation in FP64; the state is
 * Q[N][4][ML] doubles.  LXW_PREC_MIXED: FP32 bulk (point values, CK flux,
 * projections, LLF point fluxes, volume / edge integrals, shock limiter)
 * with FP64 cell averages, FP64 blended update and FP64 limiter solves where
 * an FP32 screen with an error margin cannot prove theta = 1; the state is
 * the packed layout of lxw_state_pack (averages double [4][N], their FP32
 * copy float [4][N], then higher modes float [4][ML-1][N]). */
enum { LXW_PREC_FP64 = 0, LXW_PREC_MIXED = 1 };

/* device status bits (returned in lxw_diag.status) */
enum { LXW_ST_NONPOSITIVE = 1, LXW_ST_CFL = 2, LXW_ST_NAN = 4, LXW_ST_TIMEOUT = 8 };

typedef struct lxw_mesh lxw_mesh;
typedef struct lxw_solver lxw_solver;

/* Physics and method parameters.  Defaults (lxw_options_default):
 * gamma 1.4 (Eq. eos), eps0 1e-12 (Sec. 3.1 Step 0), alpha0 500 (shock
 * limiter alpha = alpha0 * dx^1.5, Sec. 4.1), shock limiter on, FP64. */
typedef struct {
  double gamma;
  double eps0;
  double alpha0;
  int shock_limiter;
  int precision;
  int block_threads;        /* elements (threads) per CTA of the element kernels;
                               mixed form: also the tile size of the work list
                               (0 = 128; at most 128)                          */
  int ctas_per_sm;          /* mixed form: persistent CTAs per SM looping over the
                               work list (0 = one CTA per tile)                 */
  int high_occupancy;       /* mixed form: 1 = the edge and gated-shock kernels'
                               variants with more resident CTAs per SM (fewer
                               registers), faster on large meshes (0 default)  */
  int moment_exact;         /* 1 = the moment limiter's pressure step takes, per
                               point, the exact largest theta (the root of
                               rho p - eps_p rho, a quadratic in theta) instead of
                               Lemma 1's secant (Sec. 3.1 remarks it can be
                               computed exactly); never more damping (0 default) */
  int llf_global;           /* dissipation speed of the high-order point flux
                               (Eq. LLF): 0 (default) = the local Lax-Friedrichs
                               speed max(|u| + c) of the two traces at the
                               point, bounded by the global s; 1 = the global s
                               itself (the equation's literal wording).  The
                               Lax-Friedrichs flux of the cell averages always
                               uses the global s (Sec. 3.2).  With the global s
                               the paper's convergence test (Sec. 4, Table 1)
                               drops to second order; the local speed keeps
                               third order                                     */
  int ck_order;             /* order in time of the Cauchy-Kovalevskaya flux: 0 or
                               3 (default) = F + dt/2 F_t + dt^2/6 F_tt (Eq.
                               taylor3-flux); 4 adds dt^3/24 F_ttt, the next
                               term of the same series (F_ttt = F'''(q)(q_t)^3 +
                               3 F''(q)(q_t, q_tt) + F'(q) q_ttt, q_ttt = -div
                               of the projected F_tt), so that P3 elements are
                               fourth order in time too (the higher-order
                               direction of the conclusions)                   */
  int gate_scan;            /* mixed form with the learned gate: 0 (default) = the
                               plain shock kernel screens every cell, commits the
                               ones its exact screen clears and lists the rest,
                               and the gate kernel takes only the listed cells
                               (two launches); 1 = the gate kernel screens every
                               cell itself (one launch, faster on small meshes).
                               Same state either way; lxw_autotune chooses when
                               a network is attached                            */
  int reserved[3];
} lxw_options;

/* Per-step diagnostics (filled when a non-NULL pointer is passed). */
typedef struct {
  double s;                 /* global wave speed of the step (Eq. LLF)             */
  double dt;                /* time step used                                       */
  double min_rho, min_p;    /* minimum cell-average density / pressure after step  */
  double mass, momx, momy, energy;  /* sum_i |T_i| Q^(1)_i after the step          */
  double n_mom;             /* cells with moment-limiter theta < 1 (Sec. 3.1)       */
  double n_edge;            /* edges with flux-limiter theta_e < 1 (Sec. 3.3)       */
  double n_sc;              /* cells with shock-limiter theta < 1 (Sec. 4.1)        */
  int status;               /* LXW_ST_* bits seen on the device during the step     */
  int reserved;
  double n_fp64_moment;     /* mixed form: cells whose moment limiter ran in FP64   */
  double n_fp64_edge;       /* mixed form: cells whose flux-limiter solve ran in FP64 */
  double n_mlp_skip;        /* mixed form: cells the learned gate let skip the shock limiter */
} lxw_diag;

const char* lxw_last_error(void);
lxw_status lxw_options_default(lxw_options* opt);

/* --- meshes (Sec. 1.2: non-overlapping elements; Sec. 3.3: edge normals n_e
 * with |n_e| = edge length, eps_ik, owner i_e = lower element index) ----- */

/* nx*ny axis-aligned cells on [x0,x1]x[y0,y1]; element id = iy*nx + ix.
 * bc[4] = codes of the (left, right, bottom, top) sides; periodic sides
 * must be paired.  Errors: LXW_ERR_ARG. */
lxw_status lxw_mesh_cartesian(int nx, int ny, double x0, double x1, double y0, double y1,
                              const int bc[4], lxw_mesh** out);

/* The same grid without the cells whose mask_host[iy*nx + ix] is 0 (host
 * array of nx*ny bytes, read during the call; NULL keeps every cell), e.g.
 * the step of the shock-diffraction problem of Sec. 4.  Elements are the
 * kept cells numbered in row order (iy, then ix).  A face that a kept cell
 * shares with a left-out one (also across a periodic side) gets the code
 * mask_bc (REFLECT, TRANSPARENT or INFLOW).  Errors: LXW_ERR_ARG (bad code
 * or box, periodic sides unpaired, no cell kept). */
lxw_status lxw_mesh_cartesian_masked(int nx, int ny, double x0, double x1, double y0, double y1,
                                     const int bc[4], const unsigned char* mask_host, int mask_bc,
                                     lxw_mesh** out);

/* Triangles tv[nt][3] (counter-clockwise vertex ids into xy_host[nv][2]).
 * ebc_host[nt][3] (nullable; default transparent) gives the boundary code
 * (REFLECT, TRANSPARENT or INFLOW) of triangle-local edge k (vertex
 * k -> k+1), read only on boundary edges.
 * Errors: LXW_ERR_BOUNDS (vertex id), LXW_ERR_ARG (non-positive area,
 * an edge shared by more than two triangles). */
lxw_status lxw_mesh_triangles(int nv, const double* xy_host, int nt, const int* tv_host,
                              const int* ebc_host, lxw_mesh** out);
void lxw_mesh_destroy(lxw_mesh* mesh);
int lxw_mesh_num_elements(const lxw_mesh* mesh);

/* --- solver: tables, geometry and workspace on the device --------------- */

/* degree 2 or 3.  stream: cudaStream_t (NULL = legacy default stream) on
 * which every later call of this solver is enqueued.  Allocates all device
 * memory the step needs: lxw_step, lxw_run, lxw_run_host, lxw_profile_step
 * and the phase calls allocate nothing (lxw_run and lxw_profile_step
 * instantiate a CUDA graph on first use).  lxw_solver_set_mlp (the gate's
 * weight image, once), lxw_autotune (a scratch state) and lxw_step_dump
 * (a scratch theta pair) allocate as they say. */
lxw_status lxw_solver_create(const lxw_mesh* mesh, int degree, const lxw_options* opt,
                             void* stream, lxw_solver** out);
void lxw_solver_destroy(lxw_solver* s);
lxw_status lxw_solver_set_stream(lxw_solver* s, void* stream);
/* The state prim_host[4] = (rho, u, v, p) of the LXW_BC_INFLOW faces (host
 * array, read during the call; default all zero).  Outside such a face the
 * solution is that state at every point and time: its trace is q_in, the
 * time-averaged flux there n.F(q_in) (q_t = q_tt = 0), the neighbour
 * average of the limiters q_in.  The global wave speed stays the maximum
 * over the cells (Sec. 3.3).  Shared by every problem of a batched solver.
 * Drops the solver's CUDA graphs (re-captured on the next lxw_run).
 * Errors: LXW_ERR_ARG (null, rho <= 0 or p <= 0). */
lxw_status lxw_solver_set_inflow(lxw_solver* s, const double prim_host[4]);
/* N elements, E edges per element, ML modes, npts limiter points per element
 * (interior + edge quadrature points), nproj projection points. */
lxw_status lxw_solver_info(const lxw_solver* s, int* N, int* E, int* ML, int* npts, int* nproj);

/* Bytes of the solver's state buffer (N*4*ML*8 for FP64; N*4*8 + N*4*ML*4
 * for the mixed form).  lxw_state_pack converts Q64_dev[N][4][ML] doubles into
 * the solver's state layout (a copy for FP64 solvers); lxw_state_unpack
 * converts back.  Both asynchronous on the solver's stream; buffers must not
 * overlap. */
size_t lxw_state_bytes(const lxw_solver* s);
lxw_status lxw_state_pack(lxw_solver* s, const double* Q64_dev, void* state_dev);
lxw_status lxw_state_unpack(lxw_solver* s, const void* state_dev, double* Q64_dev);

/* Batch of independent problems (Sec. 1.5: problems share nothing) stepped
 * together: one solver over the disjoint union of the meshes (same element
 * kind), each problem with its own wave speed s and time step dt (Eq. LLF,
 * CFL rule).  Elements are numbered mesh 0 first, then mesh 1, ...; the
 * state is the concatenation of the problems' states in that order.  The
 * mixed form's kernels run persistent CTAs over a work list of (problem,
 * tile) pairs, so one launch per phase covers every problem and one CUDA
 * graph covers a step.  Several problems need LXW_PREC_MIXED.  Meshes may be
 * destroyed after the call. */
lxw_status lxw_batch_create(int nmesh, const lxw_mesh* const* meshes, int degree, const lxw_options* opt,
                            void* stream, lxw_solver** out);
/* Per-problem wave speed and time step of the last step (synchronises);
 * s_host / dt_host hold nprob doubles each (nullable). */
lxw_status lxw_batch_scalars(lxw_solver* s, int* nprob, double* s_host, double* dt_host);
/* Autotuner: times `reps` steps of each candidate (elements per CTA in
 * {32, 64, 128} x persistent CTAs per SM in {0 (one per tile), 1, 2, 3, 4,
 * 6, 8} x high_occupancy in {0, 1}; FP64 solvers: elements per CTA only),
 * then, with a network attached, gate_scan in {0, 1} for the fastest of those,
 * on a scratch copy of
 * state_dev (restored afterwards), keeps the fastest in the solver and
 * returns it (output pointers nullable).  Allocates a scratch state. */
lxw_status lxw_autotune(lxw_solver* s, void* state_dev, double cfl, int reps, int* block_threads,
                        int* ctas_per_sm, float* best_ms, int* high_occupancy);
/* The solver's options as it runs now (after lxw_autotune: the chosen work
 * list, variants and gate_scan).  Errors: LXW_ERR_ARG (null argument). */
lxw_status lxw_solver_get_options(const lxw_solver* s, lxw_options* out);

/* Physical coordinates of the initial-condition projection points
 * xy_host[N][nproj][2] (Gauss rule with degree+3 points per direction). */
lxw_status lxw_projection_points(const lxw_solver* s, double* xy_host);
/* Values of the modal basis phi^(l) (Sec. 1.2; the mode order of the state
 * layout above) at points of the reference element: ref_xy_host[n][2] in
 * [-1,1]^2 (quadrilaterals; x = x_c + xi dx/2, y = y_c + eta dy/2) or in
 * {xi, eta >= 0, xi + eta <= 1} (triangles; x = v0 + (v1 - v0) xi +
 * (v2 - v0) eta), written to phi_host[n][ML].  Host only, synchronous, no
 * device work: a post-processing aid (q^h at any point is sum_l Q^(l)
 * phi^(l) of the element holding it).  Errors: LXW_ERR_ARG. */
lxw_status lxw_basis_eval(int kind, int degree, int n, const double* ref_xy_host, double* phi_host);
/* L2 projection Q^(l) = (1/|T0|) Int q phi^(l) (Sec. 1.2) of primitive values
 * prim_dev[N][nproj][4] = (rho, u, v, p) at the projection points into
 * Q_dev[N][4][ML]; the energy follows Eq. eos.  Asynchronous on the stream. */
lxw_status lxw_project(lxw_solver* s, const double* prim_dev, double* Q_dev);

/* --- the hot path --------------------------------------------------------- */

/* One LxW-DG time step, in place on the state Q_dev (FP64 solvers:
 * Q[N][4][ML]; mixed solvers: the packed layout) (Sec. 3.3 Steps 1-6 and
 * the shock-capturing limiter, outline Step 5):
 *   moment limiter (Sec. 3.1) -> global wave speed s -> CK time-averaged flux
 *   and volume integral (Sec. 2.2-2.3) -> LLF edge flux, f^LxW, f^LxF (Step 3)
 *   -> flux limiter (Steps 4-5) -> blended update (Step 6) -> shock limiter.
 * dt > 0 is used as given; dt <= 0 selects dt = cfl * min_i(2|T_i|/P_i) / s.
 * theta_cell_dev (nullable) receives [2][N] = (moment theta, shock theta);
 * theta_edge_dev (nullable) receives [N][E] theta_e seen from each element.
 * diag_host (nullable) synchronises the stream and fills the diagnostics;
 * with diag_host NULL the call is asynchronous and graph-capturable.
 * Returns LXW_ERR_NONPOSITIVE / LXW_ERR_CFL / LXW_ERR_NAN / LXW_ERR_TIMEOUT
 * only when diag_host is given and the device flagged the condition during
 * this step or a step since the last diagnostics (the status bits are kept
 * until read); the steps still complete. */
lxw_status lxw_step(lxw_solver* s, double* Q_dev, double dt, double cfl, lxw_diag* diag_host,
                    double* theta_cell_dev, double* theta_edge_dev);

/* nsteps steps with dt from cfl, replayed from a CUDA graph of one step
 * captured on first use (the graph is rebuilt when Q_dev changes).  diag_host
 * (nullable) receives the last step's diagnostics. */
lxw_status lxw_run(lxw_solver* s, double* Q_dev, int nsteps, double cfl, lxw_diag* diag_host);

/* Runs steps with dt from cfl (the CFL rule, Sec. 4.1) until the state has
 * advanced by exactly t_span: the device keeps each problem's clock, takes
 * dt = min(cfl rule, t_span - t) so that the last step lands on t_span, and
 * skips a problem once its clock has reached it (each problem of a batch
 * keeps its own clock).  No host synchronisation per step: a captured graph
 * of one timed step is replayed in chunks (first one step, then as many as
 * the slowest problem needs at its mean time step so far, +5 %), with one
 * synchronisation per chunk.  At most max_steps steps.  steps_host
 * (nullable) receives the steps taken (the most over the problems),
 * t_host (nullable) the time reached (the least over the problems; t_span
 * unless max_steps stopped the run).  diag_host (nullable) receives the
 * final state's minima and conserved totals, s and dt of the last step
 * taken (largest s, smallest dt over the problems) and the status bits seen
 * since the last diagnostics; the limiter counts are zero.  Errors:
 * LXW_ERR_ARG (t_span <= 0, cfl <= 0, max_steps < 1, a batch with the
 * learned gate), LXW_ERR_CUDA, and with diag_host the device statuses of
 * lxw_step. */
lxw_status lxw_run_to(lxw_solver* s, double* Q_dev, double t_span, double cfl, int max_steps, lxw_diag* diag_host,
                      int* steps_host, double* t_host);

/* End-to-end form of lxw_run on HOST memory: brings Q_host ([N][4][ML],
 * pinned or pageable) to the solver's device state, runs nsteps and returns
 * the result to Q_host, synchronously.  Pageable memory is copied; for the
 * mixed form, pinned (device-mapped) memory is read and written directly by
 * the layout-conversion kernels, one pass over the host link each way. */
lxw_status lxw_run_host(lxw_solver* s, double* Q_host, int nsteps, double cfl, lxw_diag* diag_host);

/* The same on a HOST copy of the solver's own state layout (lxw_state_bytes
 * bytes: Q[N][4][ML] for FP64 solvers, the packed layout of lxw_state_pack
 * for mixed ones, which is 112 instead of 192 bytes per P2 cell): one
 * host-to-device copy of state_host, nsteps, one device-to-host copy back,
 * synchronously.  Pinned memory makes the copies asynchronous DMA transfers.
 * Errors: LXW_ERR_ARG, LXW_ERR_CUDA, and the device statuses of lxw_run. */
lxw_status lxw_run_host_state(lxw_solver* s, void* state_host, int nsteps, double cfl, lxw_diag* diag_host);

/* Single phases of the step, for per-phase checks (same kernels as lxw_step):
 * moment limiter on Q_dev in place (Sec. 3.1) with theta_dev[N] (nullable)
 * and the global wave speed written to s_dev[0] (device double). */
lxw_status lxw_moment_limit(lxw_solver* s, double* Q_dev, double* theta_dev, double* s_dev);
/* shock-capturing limiter (Sec. 4.1) on Q_dev in place, theta_dev[N] nullable */
lxw_status lxw_shock_limit(lxw_solver* s, double* Q_dev, double* theta_dev);

/* Number of kernel launches one lxw_step enqueues (diag_host NULL). */
int lxw_step_launches(const lxw_solver* s);
/* Number of intervals lxw_profile_step times: FP64 form one per kernel
 * (reset, moment, ck, edge, update[, shock]); mixed form 5 (moment with the
 * time step, ck, edge, update, shock with the learned gate). */
int lxw_profile_phases(const lxw_solver* s);

/* lxw_step (dt from cfl, no diagnostics) replayed from a CUDA graph with an
 * event node around each kernel (captured on first use, rebuilt when Q_dev
 * or cfl change), on the solver's stream; synchronises and writes the device
 * duration in milliseconds of each interval to ms_host[lxw_profile_phases(s)]
 * in launch order.  Tracing aid:
 * the events are created with the solver. */
lxw_status lxw_profile_step(lxw_solver* s, double* Q_dev, double cfl, float* ms_host);

/* Per-phase inspection (same kernels as lxw_step).  lxw_step_phases runs only
 * the first nphases phases of a step (1 moment limiter + wave speed, 2 CK
 * flux and volume integral, 3 edge fluxes and flux-limiter proposals,
 * 4 blended update, 5 shock limiter) in place on Q_dev.  lxw_workspace_copy
 * copies a workspace buffer to host memory after it: which = 0 edge traces
 * [E][MQ][8][N] (q then n_out.F_T at each edge point, n_out the outward
 * normal scaled by the edge length), 1 outward fluxes [E][8][N] (f^LxW then
 * f^LxF), 2 Lambda proposals [E][N], 3 wave speed and dt [2]; count = number
 * of doubles the caller's buffer holds (LXW_ERR_ARG if too small). */
lxw_status lxw_step_phases(lxw_solver* s, double* Q_dev, double dt, double cfl, int nphases);
lxw_status lxw_workspace_copy(lxw_solver* s, int which, double* host_out, size_t count);


/* --- learned troubled-cell indicator (mixed form) ------------------------
 * An MLP 24 -> 64 (ReLU) -> 64 (ReLU) -> 1 (sigmoid) predicts the theta of
 * the shock-capturing limiter (Sec. 4.1) from 24 features of a cell at the
 * limiter's input (rho and E higher modes over their averages, two momentum
 * modes over rho*(|u|+c), neighbour averages of rho and E relative to the
 * cell's, alpha/rho, the internal-energy fraction; clipped to [-8, 8]).
 * With a gate set, cells whose prediction is at least 1 - tau keep theta = 1
 * without the limiter's point work; all others run the limiter, which stays
 * the fallback.  The positivity limiters always run exactly.
 * Parameters (float, LXW_MLP_PARAMS of them): W1[24][64], b1[64],
 * W2[64][64], b2[64], w3[64], b3.  Training (FP32 kernels, mean-squared
 * error, Adam) runs on the GPU; the gated shock kernel first applies the
 * limiter's exact screen (every primitive provably within alpha of its
 * average: theta = 1), evaluates a BF16 copy of the network on the tensor
 * cores (tcgen05, FP32 accumulation in tensor memory) for the tiles of 128
 * cells that hold a cell the screen cannot clear, and runs the plain
 * limiter for the cells neither clears.  The prediction is used only for a
 * cell whose 24 features all lie inside the network's envelope (per-feature
 * bounds: those of its training data, or set explicitly); outside it the
 * limiter runs.  Its device waits are bounded (about a second): on expiry it sets
 * LXW_ST_TIMEOUT and limits the rest of its cells with the plain limiter. */
enum { LXW_MLP_IN = 24, LXW_MLP_HIDDEN = 64, LXW_MLP_PARAMS = 5825 };
typedef struct lxw_mlp lxw_mlp;
/* max_batch: largest batch of the calls below; He-initialised from seed. */
lxw_status lxw_mlp_create(int max_batch, unsigned long long seed, void* stream, lxw_mlp** out);
void lxw_mlp_destroy(lxw_mlp* n);
int lxw_mlp_num_params(void);
lxw_status lxw_mlp_get_params(lxw_mlp* n, float* params_dev);
lxw_status lxw_mlp_set_params(lxw_mlp* n, const float* params_dev);
/* yhat_dev[B] = network(X_dev[B][24]) */
lxw_status lxw_mlp_forward(lxw_mlp* n, const float* X_dev, int B, float* yhat_dev);
/* mean-squared error on (X_dev[B][24], y_dev[B]) and its gradient
 * grad_dev[LXW_MLP_PARAMS] (nullable); loss_host nullable (synchronises). */
lxw_status lxw_mlp_loss_grad(lxw_mlp* n, const float* X_dev, const float* y_dev, int B, float* loss_host,
                             float* grad_dev);
/* epochs of Adam over shuffled mini-batches (seeded) of the count samples.
 * Also widens the envelope to the per-feature range of X_dev (the first
 * call on a network, or after lxw_mlp_set_envelope(n, NULL, NULL), sets it). */
lxw_status lxw_mlp_train(lxw_mlp* n, const float* X_dev, const float* y_dev, int count, int epochs, int batch,
                         float lr, unsigned long long seed, float* last_loss);
/* The envelope: lo_host[24] <= feature <= hi_host[24] is where the gate
 * uses the prediction.  Both NULL: unbounded (a new network's default; the
 * next training call sets the envelope).  Takes effect at the next
 * lxw_solver_set_mlp.  Errors: LXW_ERR_ARG (one NULL, lo > hi). */
lxw_status lxw_mlp_set_envelope(lxw_mlp* n, const float* lo_host, const float* hi_host);
/* Copies the current envelope into lo_host[24], hi_host[24] (-inf / +inf
 * where unbounded).  Errors: LXW_ERR_ARG (null argument). */
lxw_status lxw_mlp_get_envelope(const lxw_mlp* n, float* lo_host, float* hi_host);
/* Enables (mlp non-NULL) or disables the learned gate of a mixed solver;
 * the solver keeps a BF16 copy taken now, laid out as the tensor-core
 * operands (later training needs another call).  tau in [0, 1).  Errors:
 * LXW_ERR_ARG (FP64 solver, tau), LXW_ERR_CUDA. */
lxw_status lxw_solver_set_mlp(lxw_solver* s, lxw_mlp* mlp, float tau);
/* Test aid of the gate's bounded device waits (no counterpart in the
 * paper): with cycles > 0, every CTA of the gated shock kernel, at its first
 * tile that needs the network, first waits at most `cycles` SM cycles on
 * its own MMA barrier before anything was committed to it.  Nothing can
 * arrive there, so the wait runs out and the CTA takes the timeout path:
 * LXW_ST_TIMEOUT (LXW_ERR_TIMEOUT from the next step with diagnostics), the
 * plain shock limiter on all its cells (the state equals the ungated step's),
 * the weight copy still awaited with the normal bound, tensor memory
 * released.  0 (default) switches it off.  Drops the solver's CUDA graphs.
 * Errors: LXW_ERR_ARG (null solver, cycles < 0). */
lxw_status lxw_solver_set_gate_wait_test(lxw_solver* s, long long cycles);

/* One mixed step (plain limiter, no gate) that also writes each cell's
 * features at the shock limiter's input (feat_dev[N][24]; rows of cells with
 * non-positive new averages are left untouched) and the limiter's theta
 * (theta_sc_dev[N], nullable): training pairs produced by the method itself.
 * Synchronous; allocates a scratch theta pair when theta_sc_dev is given.
 * Errors: LXW_ERR_ARG (FP64 form, shock limiter off), LXW_ERR_CUDA. */
lxw_status lxw_step_dump(lxw_solver* s, void* state_dev, double cfl, float* feat_dev, double* theta_sc_dev);

/* One mixed step gated by the solver's network (lxw_solver_set_mlp), that
 * also writes the network's output theta_hat for every cell
 * (gate_dev[N], FP32; NaN where the cell's new averages are not positive,
 * so that the limiter runs without asking the network) and, when feat_dev
 * is not null, the cell's features (feat_dev[N][24]).  The network runs on
 * the tensor cores: BF16 features and weights, FP32 accumulation, the
 * hidden layer rounded to BF16 between the two matrix products, FP32
 * output layer and sigmoid.  Errors: LXW_ERR_ARG (null pointer, FP64
 * form, shock limiter off, no network), LXW_ERR_CUDA. */
lxw_status lxw_step_gate(lxw_solver* s, void* state_dev, double cfl, float* gate_dev, float* feat_dev);

/* Allocation-free form of lxw_moment_limit, for callers that cannot call
 * cudaMalloc: code whose device memory is owned by another allocator (a
 * framework's caching pool, or a fixed budget set aside at start-up, where
 * an extra allocation could fail or fragment it), and code that must avoid
 * cudaMalloc's implicit device synchronisation.  The paper has no
 * counterpart; it is the same moment limiter and wave-speed maximum,
 * without a solver.
 * Q_dev[n_elements][4][ML] is limited in place; theta_dev[n_elements]
 * (nullable) receives theta; s_dev[0] (device double) receives the wave
 * speed.  No geometry is needed (the limiter is element-local).
 * Status: a cell whose input average has rho <= 0 or p <= 0 keeps its
 * average, gets theta = 0 and has its higher modes zeroed, and sets
 * LXW_ST_NONPOSITIVE.  With status_dev (device unsigned int, nullable) the
 * call is asynchronous on `stream` and the device writes the LXW_ST_* bits
 * of this call there; with status_dev NULL the call waits for `stream` and
 * returns LXW_ERR_NONPOSITIVE when the bit is set.
 * Scratch: the reduction's running maxima and the status word live in a
 * static device array of 513 64-bit words (about 4 KB) that every GPU
 * loading the library holds until exit; n_elements above 16,777,216 (512
 * slots x 32,768 elements) is rejected with LXW_ERR_ARG.  The array is
 * shared by every call and keeps the last call's contents; each call clears
 * the slots it uses and the status word first.  Calls that overlap on the
 * GPU (concurrent streams, or several host threads) race on it and must be
 * serialised by the caller.  The first call on a device finds the array's
 * device address and loads the basis tables into the constant bank (once
 * per device, with that device current); make that first call before any
 * stream capture.  Allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library call.  A CUDA error already pending on the calling
 * thread is reported (LXW_ERR_CUDA) and left in place; nothing is launched.
 * Errors: LXW_ERR_ARG (null pointer, kind/degree, size, gamma <= 1,
 * eps0 <= 0), LXW_ERR_CUDA, LXW_ERR_NONPOSITIVE (status_dev NULL only). */
lxw_status lxw_moment_limit_noalloc(int kind, int degree, int n_elements, double gamma, double eps0,
                                    double* Q_dev, double* theta_dev, double* s_dev, unsigned int* status_dev,
                                    void* stream);

/* ------------------------------------------------------------------ */
/* 3D Cartesian meshes (hexahedra): the same step on box cells with six    */
/* faces (the extension the end of Sec. 3.3 says carries over directly;   */
/* the 3D Euler equations of Sec. 1.1 with a third flux H), in FP64 or in */
/* the mixed form (options.precision; see lxw3_solver_create).            */
/* State Q[N][5][ML] (rho, rho u, rho v, rho w, E), ML = 4 (P1) or 10      */
/* (P2); cell (ix, iy, iz) is element (iz ny + iy) nx + ix; modes           */
/* L_a(xi) L_b(eta) L_c(zeta), L_n = sqrt(2n+1) P_n, a + b + c <= degree,  */
/* ordered by total degree, then a descending, then b descending (the     */
/* cell average is mode 0).  Faces and sides are ordered x-, x+, y-, y+,   */
/* z-, z+.  Readings beyond the 2D step: dt = cfl * hmin / s with hmin =    */
/* 3 |K| / |dK| (half the cell side, as in 2D); the shock limiter's alpha  */
/* = alpha0 * (|K|^(1/3))^1.5; the flux limiter gives every face with a     */
/* negative density difference the same Lambda and takes mu over the 63    */
/* corners of the box of the six proposals.                                */
/* ------------------------------------------------------------------ */
typedef struct lxw_solver3 lxw_solver3;

typedef struct {
  double s, dt;               /* global wave speed and time step of the step       */
  double min_rho, min_p;      /* minimum cell-average density / pressure after it  */
  double mass, momx, momy, momz, energy;   /* sum_i |K_i| Q^(1)_i after the step   */
  double n_mom;               /* cells with moment-limiter theta < 1                */
  double n_face;              /* faces with flux-limiter theta < 1                  */
  double n_sc;                /* cells with shock-limiter theta < 1                 */
  int status;                 /* LXW_ST_* bits of the step                          */
  int reserved;
} lxw_diag3;

/* nx x ny x nz cells of box = (x0, x1, y0, y1, z0, z1); bc[6] per side:
 * LXW_BC_PERIODIC (paired on both sides of an axis), LXW_BC_REFLECT or
 * LXW_BC_TRANSPARENT.  degree 1 or 2.  Options: gamma, eps0, alpha0,
 * shock_limiter, llf_global, block_threads, precision; moment_exact 0 and
 * ck_order 3 (or 0).  precision LXW_PREC_FP64: every operation in FP64;
 * LXW_PREC_MIXED: the Cauchy-Kovalevskaya kernel (point values, flux
 * derivatives, q_t and q_tt, the volume integral, the traces) in FP32,
 * while the state, the cell averages, the face fluxes, the moment, flux and
 * shock limiters and every positivity decision stay FP64 (the state keeps
 * its FP64 layout; the volume term is added to it in FP64).  Allocates the
 * workspace (about (60 NF + 90) doubles per cell, NF = (degree + 1)^2).
 * Errors: LXW_ERR_ARG, LXW_ERR_NOMEM, LXW_ERR_CUDA. */
lxw_status lxw3_solver_create(int nx, int ny, int nz, const double box[6], const int bc[6], int degree,
                              const lxw_options* opt, void* stream, lxw_solver3** out);
void lxw3_solver_destroy(lxw_solver3* s);
/* cells, modes per variable, projection points per cell (nullable outputs) */
lxw_status lxw3_solver_info(const lxw_solver3* s, int* n_elements, int* n_modes, int* n_proj_points);
/* physical coordinates xyz_host[N][NPJ][3] of the projection points */
lxw_status lxw3_projection_points(const lxw_solver3* s, double* xyz_host);
/* Q_dev[N][5][ML] = L2 projection of prim_dev[N][NPJ][5] = (rho, u, v, w, p) */
lxw_status lxw3_project(lxw_solver3* s, const double* prim_dev, double* Q_dev);
/* One step in place (dt > 0 fixes dt, else dt = cfl * hmin / s); fills
 * diag_host (nullable), theta_face_dev[N][E] (nullable; E = 6 on
 * hexahedra, 4 on tetrahedra); synchronises.
 * Returns LXW_ERR_NONPOSITIVE / LXW_ERR_CFL / LXW_ERR_NAN from the step's
 * status bits (the step itself completes). */
lxw_status lxw3_step(lxw_solver3* s, double* Q_dev, double dt, double cfl, lxw_diag3* diag_host,
                     double* theta_face_dev);
/* nsteps CFL steps: the first nsteps - 1 replay one captured CUDA graph (no
 * host synchronisation), the last runs as lxw3_step and reports. */
lxw_status lxw3_run(lxw_solver3* s, double* Q_dev, int nsteps, double cfl, lxw_diag3* diag_host);
/* one step timed per phase: ms[5] = moment, ck, face, update, shock */
lxw_status lxw3_profile_step(lxw_solver3* s, double* Q_dev, double cfl, float* ms);
/* kernel launches of one step without diagnostics */
int lxw3_step_launches(const lxw_solver3* s);

/* Tetrahedral meshes, FP64: the same step on unstructured cells with four
 * faces, through the same solver type and the lxw3_step / lxw3_run /
 * lxw3_project / lxw3_profile_step calls above (theta_face_dev is then
 * [N][4]).  Each cell is the affine image of the reference tetrahedron
 * T0 = {r, s, t >= 0, r + s + t <= 1} taking T0's vertices (0,0,0),
 * (1,0,0), (0,1,0), (0,0,1) to the cell's vertices 0..3 in the order given.
 * Modes: the orthonormal basis (under (1/|K|) Int) obtained by Gram-Schmidt
 * from the monomials r^a s^b t^c in the mode order of the hexahedra (mode 0
 * = 1, the cell average).  Interior quadrature: a conical product of
 * Gauss-Jacobi rules with degree + 1 points per direction; face k (opposite
 * vertex k): a collapsed triangle rule with (degree + 1)^2 points placed from
 * the face's vertices in ascending vertex-id order, so both cells of a face
 * meet the same points in the same order.  Both rules integrate total
 * degree 2 degree + 1 exactly.
 *   xyz[n_vertices][3] (host): vertex positions;
 *   tets[n_tets][4] (host): vertex indices, positively oriented (the
 *     determinant of (x1 - x0, x2 - x0, x3 - x0) is positive);
 *   vid[n_vertices] (host): vertex ids; two faces with the same three ids
 *     are glued (periodic images carry equal ids; give vid[v] = v for an
 *     ordinary mesh).  A cell's four ids must differ;
 *   face_bc[n_tets][4] (host, nullable = all transparent): the code of face
 *     k of each cell, read only where no other cell has its ids:
 *     LXW_BC_REFLECT or LXW_BC_TRANSPARENT.
 * dt = cfl * hmin / s with hmin = min 3 |K| / |dK| over the cells; the shock
 * limiter's alpha = alpha0 * (|K|^(1/3))^1.5 per cell; the flux limiter's mu
 * runs over the 15 corners of the box of four proposals.  The host arrays
 * are read during the call only.  Allocates about (40 NF + 90) doubles per
 * cell of workspace plus 26 doubles and 5 ints of geometry.  Errors:
 * LXW_ERR_ARG (null pointer, sizes, degree, index out of range, repeated id
 * in a cell, non-positive orientation, a face shared by more than two
 * cells, a bad boundary code), LXW_ERR_NOMEM, LXW_ERR_CUDA. */
lxw_status lxw3_solver_create_tets(int n_vertices, const double* xyz, int n_tets, const int* tets, const int* vid,
                                   const int* face_bc, int degree, const lxw_options* opt, void* stream,
                                   lxw_solver3** out);
/* faces per element: 6 (hexahedra) or 4 (tetrahedra); 0 for NULL */
int lxw3_faces_per_element(const lxw_solver3* s);

#ifdef __cplusplus
}
#endif
#endif
