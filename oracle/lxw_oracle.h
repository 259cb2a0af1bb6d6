/*
 * lxw_oracle.h -- plain FP64 CPU oracle of the positivity-preserving
 * Lax-Wendroff DG time step for the 2D Euler equations.
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle exists to check the GPU library; it
 * shares no code, header, table or constant generator with it.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark load
 * it.  It is written for clarity, one element or one edge at a time, in the
 * order the paper presents the method:
 *   Sec. 3.1  moment limiter (Steps 0-2, Lemma 1)
 *   Sec. 2.2  Cauchy-Kovalevskaya time-averaged flux, Eqs. fluxderivs-a/b,
 *             taylor3-flux
 *   Sec. 2.3  fully discrete weak form (Steps 1-4), Eq. EulerStepExactGalerkin,
 *             local Lax-Friedrichs flux Eq. LLF
 *   Sec. 2.4  reflective / transparent boundary states
 *   Sec. 3.2-3.3  parameterised flux limiter (Steps 3-6)
 *   Sec. 4.1  shock-capturing limiter applied after the update
 *
 * Conventions shared with the GPU library by documentation only (no code):
 *   state layout Q[N][4][ML], variables (rho, rho*u, rho*v, E), mode order
 *   documented in lxw_oracle.c; boundary codes 0 periodic, 1 reflective,
 *   2 transparent, 3 inflow (the solver's prescribed state); element kinds
 *   0 quadrilateral (axis-aligned), 1 triangle.
 */
#ifndef LXW_ORACLE_H
#define LXW_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_mesh orc_mesh;
typedef struct orc_solver orc_solver;

/* diagnostics written by orc_step (indices into a double[ORC_DIAG_LEN]) */
enum {
  ORC_D_S = 0, ORC_D_DT, ORC_D_MINRHO, ORC_D_MINP, ORC_D_MASS, ORC_D_MOMX,
  ORC_D_MOMY, ORC_D_ENERGY, ORC_D_NMOM, ORC_D_NEDGE, ORC_D_NSC, ORC_D_STATUS,
  ORC_DIAG_LEN = 16
};
/* status bits */
enum { ORC_ST_NONPOSITIVE = 1, ORC_ST_CFL = 2, ORC_ST_NAN = 4 };

/* Gauss-Legendre rule on [-1,1] (weights sum to 2), ascending nodes. */
void orc_gauss_legendre(int n, double* x, double* w);

/* Basis: number of modes for (kind, degree). */
int orc_num_modes(int kind, int deg);
/* Orthonormal modal basis and its reference gradient at npts points. */
int orc_basis_eval(int kind, int deg, int npts, const double* xi, const double* eta,
                   double* phi, double* dphi_dxi, double* dphi_deta);
/* Interior rule with n points per direction; weights sum to 1. */
int orc_interior_rule(int kind, int n, double* xi, double* eta, double* w);

/* Euler flux F (x) and G (y) of q, and its first / second directional
 * derivatives along w (Eqs. 1-2, fluxderivs-a/b). */
void orc_flux(double gamma, const double* q, double* F, double* G);
void orc_flux_d1(double gamma, const double* q, const double* w, double* F1, double* G1);
void orc_flux_d2(double gamma, const double* q, const double* w, double* F2, double* G2);
/* third directional derivative of (F, G) along w (fourth-order CK term) */
void orc_flux_d3(double gamma, const double* q, const double* w, double* F3, double* G3);
/* mixed second derivative of (F, G) in the directions a and b */
void orc_flux_d11(double gamma, const double* q, const double* a, const double* b, double* F2, double* G2);

/* Meshes. bc[4] = (left, right, bottom, top). Triangles must be CCW;
 * ebc[nt][3] gives the boundary code of each triangle-local edge k (from
 * vertex k to vertex k+1), used only on boundary edges; NULL = transparent. */
orc_mesh* orc_mesh_cartesian(int nx, int ny, double x0, double x1, double y0, double y1,
                             const int* bc);
orc_mesh* orc_mesh_triangles(int nv, const double* xy, int nt, const int* tv, const int* ebc);
void orc_mesh_free(orc_mesh* m);
int orc_mesh_num_elements(const orc_mesh* m);
int orc_mesh_num_edges(const orc_mesh* m);
int orc_mesh_edges_per_element(const orc_mesh* m);
/* per element: area, perimeter, centroid (x,y) */
void orc_mesh_geometry(const orc_mesh* m, double* area, double* perim, double* cx, double* cy);

orc_solver* orc_solver_new(const orc_mesh* m, int deg, double gamma);
void orc_solver_free(orc_solver* s);
void orc_solver_set_params(orc_solver* s, double eps0, double alpha0, int shock_limiter);
/* 1: the moment limiter's pressure step by the exact root (Sec. 3.1 remark), 0: secant */
void orc_solver_set_moment_exact(orc_solver* s, int flag);
/* flag 1: the high-order point flux (Eq. LLF) dissipates with the global s
 * instead of the local speed of its two traces (default 0) */
void orc_solver_set_llf_global(orc_solver* s, int flag);
/* CK time order: 3 (default, Eq. taylor3-flux) or 4; returns 1 otherwise */
int orc_solver_set_ck_order(orc_solver* s, int order);
/* state of the inflow boundaries, primitive (rho, u, v, p) */
void orc_solver_set_inflow(orc_solver* s, const double* prim);
/* Cartesian mesh without the cells of mask == 0 (mask[ny][nx], row order);
 * faces towards a left-out cell get the code mask_bc */
orc_mesh* orc_mesh_cartesian_masked(int nx, int ny, double x0, double x1, double y0, double y1, const int* bc,
                                    const unsigned char* mask, int mask_bc);
int orc_solver_num_modes(const orc_solver* s);
int orc_solver_num_points(const orc_solver* s);   /* interior + edge points per element */
int orc_projection_num_points(const orc_solver* s);
void orc_projection_points(const orc_solver* s, double* xy);   /* [N][np][2] */
void orc_projection_weights(const orc_solver* s, double* w);   /* [np], sum 1 */
void orc_project(const orc_solver* s, const double* prim, double* Q); /* prim[N][np][4] */
void orc_eval_projection_points(const orc_solver* s, const double* Q, double* q); /* [N][np][4] */
/* state at the limiter points (interior then edge points) [N][npts][4] */
void orc_eval_limiter_points(const orc_solver* s, const double* Q, double* q);
/* physical coordinates of the limiter points [N][npts][2] */
void orc_limiter_points(const orc_solver* s, double* xy);
/* After orc_step: per element edge the outward f^LxW and f^LxF [N][E][4]
 * (eps_ik applied) and the dt used. */
double orc_last_fluxes(const orc_solver* s, double* fw, double* ff);

/* Single phases (used by the tests to pin each part). */
double orc_moment_limit(const orc_solver* s, double* Q, double* theta, int* status);
double orc_wave_speed(const orc_solver* s, const double* Q);
/* CK time-averaged flux at all points of element i for a given dt:
 * outputs per point (interior then edge points) q, q_t, q_tt, F_T, G_T [npts][4]. */
void orc_ck_element(const orc_solver* s, const double* Q, int i, double dt, double* q,
                    double* qt, double* qtt, double* FT, double* GT, double* V);
double orc_mu_solve(double gamma, double eps0, const double* qlxf, const double* qc);
/* Flux limiter of one element (Steps 4-5) from outward fluxes fW, fF [E][4];
 * writes the Lambda proposals prop[E]; returns 1 when Gamma^rho < 0. */
int orc_flux_limit_cell(double gamma, double eps0, int E, double area, double dt, const double* qbar,
                        const double* fW, const double* fF, double* prop);
void orc_shock_limit(const orc_solver* s, double* Q, double* theta);

/* One full time step (rows a1..a10). dt_in <= 0 selects dt from cfl.
 * theta_mom[N], theta_sc[N], theta_edge[N][E] may be NULL. Returns status. */
int orc_step(orc_solver* s, double* Q, double dt_in, double cfl, double* diag,
             double* theta_mom, double* theta_sc, double* theta_edge);
/* Learned indicator: FP64 MLP 24 -> 64 -> 64 -> 1 (ReLU, ReLU, sigmoid),
 * parameters W1[24][64], b1[64], W2[64][64], b2[64], w3[64], b3.  Returns
 * the mean-squared error on (X[B][24], y[B]) (y NULL: no loss) and writes
 * the gradient (nullable) and predictions (nullable). */
double orc_mlp_loss_grad(const double* P, const double* X, const double* y, int B, double* grad, double* yhat);
/* The indicator's 24 features of every cell of Q [N][24]. */
void orc_features(const orc_solver* s, const double* Q, double* F);
/* Number of OpenMP threads the oracle uses (1 without OpenMP). */
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
