/*
 * lxw_oracle3d.h -- plain FP64 CPU oracle of the same positivity-preserving
 * Lax-Wendroff DG time step on 3D meshes of hexahedra (Cartesian) and
 * tetrahedra, the extension the paper states carries over directly (end of Sec. 3.3; the
 * 3D Euler equations of Sec. 1.1 with a third flux H).
 *
 * TEST INFRASTRUCTURE ONLY.  Like the 2D oracle it shares no code, header,
 * table or constant generator with the GPU library, and only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg load it.  It follows
 * the 2D oracle's step element by element and face by face:
 *   Sec. 3.1  moment limiter (Steps 0-2, Lemma 1, secant form)
 *   Sec. 2.2  Cauchy-Kovalevskaya time-averaged flux F_T = F + dt/2 F_t +
 *             dt^2/6 F_tt for the three flux directions
 *   Sec. 2.3  weak form, Eq. LLF with the local speed of the two traces
 *             (reading L0; the global s with llf_global)
 *   Sec. 2.4  reflective / transparent / periodic sides
 *   Sec. 3.2-3.3  flux limiter with E faces (6 on a hexahedron, 4 on a
 *             tetrahedron): Lambda from the density (Step 4), mu over the
 *             2^E - 1 corners of the box (Step 5)
 *   Sec. 4.1  shock limiter on (rho, u, v, w, p) with the E face neighbours
 *
 * Conventions, shared with the GPU library by documentation only:
 *   state Q[N][5][ML], variables (rho, rho u, rho v, rho w, E);
 *   hexahedra: cell (ix, iy, iz) is element (iz * ny + iy) * nx + ix;
 *   faces k = 0..5: x-, x+, y-, y+, z-, z+; bc[6] per domain side in that
 *   order (0 periodic, 1 reflective, 2 transparent);
 *   modes (a, b, c) with a + b + c <= deg, ordered by total degree, then a
 *   descending, then b descending; phi = L_a(xi) L_b(eta) L_c(zeta) with
 *   L_n = sqrt(2n + 1) P_n on [-1, 1] (orthonormal under (1/8) Int);
 *   points: the (deg+1)^3 interior Gauss points (xi fastest), then face k's
 *   (deg+1)^2 Gauss points at NQ + k * NF + (s + n t), s and t the two
 *   tangential directions in x, y, z order, each ascending -- so the two
 *   cells of a face see its points in the same order.
 * Tetrahedra: the reference cell T0 = {r, s, t >= 0, r + s + t <= 1}, mapped
 *   affinely from the cell's vertices 0..3; the basis is the Gram-Schmidt
 *   orthonormalisation (under (1/|T0|) Int, in the mode order above) of the
 *   monomials r^a s^b t^c; interior points a collapsed (Duffy) Gauss rule
 *   with deg + 2 points per direction, face points a collapsed triangle rule
 *   with deg + 1 per direction, placed from the face's three vertices taken
 *   in ascending vertex-id order, so again both cells see the same points in
 *   the same order.
 */
#ifndef LXW_ORACLE3D_H
#define LXW_ORACLE3D_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc3_mesh orc3_mesh;
typedef struct orc3_solver orc3_solver;

/* diagnostics written by orc3_step (indices into a double[ORC3_DIAG_LEN]) */
enum {
  ORC3_D_S = 0, ORC3_D_DT, ORC3_D_MINRHO, ORC3_D_MINP, ORC3_D_MASS, ORC3_D_MOMX, ORC3_D_MOMY,
  ORC3_D_MOMZ, ORC3_D_ENERGY, ORC3_D_NMOM, ORC3_D_NFACE, ORC3_D_NSC, ORC3_D_STATUS,
  ORC3_DIAG_LEN = 16
};

int orc3_num_modes(int deg);
/* exponents (a, b, c) of mode l */
void orc3_mode_exponents(int deg, int* abc);
/* basis and its reference gradient at npts points (outputs [npts][ML], nullable) */
int orc3_basis_eval(int deg, int npts, const double* xi, const double* eta, const double* zeta, double* phi,
                    double* dxi, double* deta, double* dzeta);

/* Euler flux of q (5 values): F[3][5] for the x, y, z directions. */
void orc3_flux(double gamma, const double* q, double* F);
/* Taylor coefficients of F(q(t)), q(t) = sum_k qs[k] t^k (k = 0..K, K <= 3):
 * Fs[k][3][5].  Coefficient 1 of q + t w is F'(q) w; twice coefficient 2 of
 * q + t a + t^2 b / 2 is F''(q)(a, a) + F'(q) b. */
void orc3_flux_series(double gamma, int K, const double* qs, double* Fs);

orc3_mesh* orc3_mesh_cartesian(int nx, int ny, int nz, const double* box, const int* bc);
/* Tetrahedra: vertex positions xyz[nv][3], cells tets[nt][4] (positively
 * oriented), vertex ids vid[nv] that identify periodic images (faces match
 * by their sorted ids), fbc[nt][4] boundary codes of the faces opposite each
 * vertex (used on unmatched faces; NULL = transparent).  Face k of a cell
 * is the one opposite its vertex k; its points come from its vertices in
 * ascending id order.  NULL on bad input. */
orc3_mesh* orc3_mesh_tets(int nv, const double* xyz, int nt, const int* tets, const int* vid, const int* fbc);
int orc3_mesh_faces_per_element(const orc3_mesh* m);
/* the tetrahedral basis (Gram-Schmidt of the monomials on the reference
 * tetrahedron, orthonormal under (1/|T0|) Int) and its gradient */
int orc3_tet_basis_eval(int deg, int npts, const double* r, const double* s, const double* t, double* phi,
                        double* dr, double* ds, double* dt);
void orc3_mesh_free(orc3_mesh* m);
int orc3_mesh_num_elements(const orc3_mesh* m);
/* per element: volume and centroid */
void orc3_mesh_geometry(const orc3_mesh* m, double* vol, double* cx, double* cy, double* cz);

orc3_solver* orc3_solver_new(const orc3_mesh* m, int deg, double gamma);
void orc3_solver_free(orc3_solver* s);
void orc3_solver_set_params(orc3_solver* s, double eps0, double alpha0, int shock_limiter);
void orc3_solver_set_llf_global(orc3_solver* s, int flag);
int orc3_solver_num_modes(const orc3_solver* s);
int orc3_solver_num_points(const orc3_solver* s);
int orc3_projection_num_points(const orc3_solver* s);
/* physical coordinates [N][NPJ][3] of the projection points and their weights [NPJ] */
void orc3_projection_points(const orc3_solver* s, double* xyz);
void orc3_projection_weights(const orc3_solver* s, double* w);
/* L2 projection of primitive values prim[N][NPJ][5] = (rho, u, v, w, p) */
void orc3_project(const orc3_solver* s, const double* prim, double* Q);
void orc3_eval_projection_points(const orc3_solver* s, const double* Q, double* q);
/* limiter points (interior + faces): coordinates [N][NPT][3], values [N][NPT][5] */
void orc3_limiter_points(const orc3_solver* s, double* xyz);
void orc3_eval_limiter_points(const orc3_solver* s, const double* Q, double* q);

/* Sec. 3.1 on every element; returns min theta; theta[N] nullable */
double orc3_moment_limit(const orc3_solver* s, double* Q, double* theta, int* status);
/* global wave speed: max |u| + c over averages and limiter points */
double orc3_wave_speed(const orc3_solver* s, const double* Q);
/* CK on element i: q, qt, qtt [NPT][5], FT [NPT][3][5], V [ML][5] (nullable) */
void orc3_ck_element(const orc3_solver* s, const double* Q, int i, double dt, double* q, double* qt,
                     double* qtt, double* FT, double* V);
/* Sec. 3.3 Steps 4-5 on one cell with E faces: prop[E]; returns 1 if Gamma^rho < 0 */
int orc3_flux_limit_cell(double gamma, double eps0, int E, double vol, double dt, const double* qbar,
                         const double* fW, const double* fF, double* prop);
double orc3_mu_solve(double gamma, double eps0, const double* ql, const double* qc);
/* Sec. 4.1 on every element; theta[N] nullable */
void orc3_shock_limit(const orc3_solver* s, double* Q, double* theta);
/* one step; dt_in > 0 fixes dt, else dt = cfl * hmin / s.  diag[ORC3_DIAG_LEN],
 * theta_mom[N], theta_sc[N], theta_face[N][E] nullable.  Returns status bits
 * (1 non-positive input average, 2 Gamma^rho < 0, 4 NaN). */
int orc3_step(orc3_solver* s, double* Q, double dt_in, double cfl, double* diag, double* theta_mom,
              double* theta_sc, double* theta_face);
/* f^LxW and f^LxF of the last step per element face, outward: [N][E][5]; returns dt */
double orc3_last_fluxes(const orc3_solver* s, double* fw, double* ff);

#ifdef __cplusplus
}
#endif
#endif
