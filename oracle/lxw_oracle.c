/*
 * lxw_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see the
 * header).  Every function cites the passage of the paper it follows.
 * Built with -ffp-contract=off so that each operation is rounded once.
 *
 * Readings of passages the paper leaves open (listed again in the design
 * notes of the repository):
 *  - weak-form signs: Q^(l) += dt/|T| (Int grad(phi).F_T - Oint phi F*.n)
 *    (integration by parts of Eq. taylor3; consistent with the l=1 update).
 *  - F_tt = F''(q)(q_t,q_t) + F'(q) q_tt with q_t = -div F^h and
 *    q_tt = -div (F_t)^h taken of the projected expansions (Sec. 2.3 Step 2).
 *  - Moment limiter secant: theta_m = theta_rho (p0 - eps_p)/(p0 - p^{theta_rho}_m)
 *    where p^{theta_rho}_m < eps_p (Lemma 1 with the density factor), floors
 *    eps_rho = min(eps0, rho_avg/2), eps_p = min(eps0, p_avg/2).  Optional
 *    variant (the exact computation Sec. 3.1 mentions): theta_m = the root in
 *    (0, theta_rho) of rho p - eps_p rho along the limited state, a quadratic.
 *  - Density flux limiter: every edge with a negative density flux
 *    difference gets the same Lambda = (Gamma^rho - |T| eps/dt)/|sum of the
 *    negative ones|, clipped to [0,1] (the four cases of Step 4, extended to
 *    4 edges, with the floor eps = min(eps0, rho^LxF/2)).
 *  - Corner states of Step 5(a) include the LxF flux on the edges with
 *    alpha_k = 0, i.e. they are the corners of the box [0,Lambda].
 *  - mu_c is the largest mu in [0,1] with p >= min(eps0, p^LxF/2) (exact
 *    root of the quadratic rho*p along the segment).
 *  - global wave speed s = max over averages and limited point values of
 *    |u| + c, computed once per step after the moment limiter; it sets dt
 *    and the Lax-Friedrichs flux f^LxF of the cell averages (Sec. 3.2: the
 *    global speed is what makes that flux positivity preserving).
 *  - the dissipation of the high-order point flux (Eq. LLF) is the local
 *    Lax-Friedrichs speed of the two traces at the point, max(|u|+c) of q-
 *    and q+, never above the global s (which bounds it in exact arithmetic:
 *    the edge points are among the limited points).  With the global s in
 *    that term as well, the paper's own convergence test (Sec. 4, Table 1)
 *    falls to second order; the local speed gives third order.  The literal
 *    global reading stays available (orc_solver_set_llf_global).
 *  - dt = cfl * min_i(2|T_i|/P_i) / s.
 *  - optional fourth order in time (ck_order 4): the next term of the Taylor
 *    series of the time-averaged flux, dt^3/24 F_ttt with F_ttt =
 *    F'''(q)(q_t,q_t,q_t) + 3 F''(q)(q_t,q_tt) + F'(q) q_ttt and
 *    q_ttt = -div F_tt^h of the projected F_tt (as for q_t and q_tt).
 *  - the shock-capturing limiter of Sec. 4.1 (cited, not printed) is read
 *    as: for w in (rho,u,v,p), M = max(w_i + alpha, max_j w_j),
 *    m = min(w_i - alpha, min_j w_j) over face neighbours j,
 *    theta_w = min(1, (M - w_i)/(max_pts w - w_i), (w_i - m)/(w_i - min_pts w)),
 *    theta_sc = min_w theta_w, alpha = alpha0 * dx^1.5, applied to all
 *    higher moments of the conserved variables.  Pinned on the density
 *    (where only the density varies over a cell, theta_sc equals its ratio
 *    and the limited density touches its bound); its agreement with the
 *    cited method itself is parity unpinned.
 *
 * Mode order.  Quadrilateral [-1,1]^2 (total degree <= deg, tensor Legendre
 * products normalised so that (1/4) Int phi_k phi_l = delta_kl):
 *   P2: 1, L1(x), L1(y), L1(x)L1(y), L2(x), L2(y)
 *   P3: ... , L3(x), L2(x)L1(y), L1(x)L2(y), L3(y)
 * Triangle {x,y >= 0, x+y <= 1}: Gram-Schmidt of the monomials
 *   1, x, y, x^2, xy, y^2, x^3, x^2 y, x y^2, y^3
 * under (1/|T0|) Int over the triangle, using the exact integrals
 *   Int x^a y^b = a! b! / (a+b+2)!.
 */
#include "lxw_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 4
#define MAXML 10
#define MAXQ 64     /* interior points */
#define MAXMQ 8     /* points per edge */
#define MAXE 4
#define MAXPTS (MAXQ + MAXE * MAXMQ)
#define MAXPJ 64    /* projection points */

enum { BC_PERIODIC = 0, BC_REFLECT = 1, BC_TRANSPARENT = 2, BC_INFLOW = 3 };
enum { KIND_QUAD = 0, KIND_TRI = 1 };

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Quadrature: Gauss-Legendre by Newton iteration on P_n.              */
/* ------------------------------------------------------------------ */
static void legendre_pn(int n, double z, double* pn, double* dpn) {
  double p0 = 1.0, p1 = z;
  if (n == 0) { *pn = 1.0; *dpn = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
    p0 = p1; p1 = p2;
  }
  *pn = p1;
  *dpn = n * (z * p1 - p0) / (z * z - 1.0);
}

void orc_gauss_legendre(int n, double* x, double* w) {
  /* roots of P_n in ascending order, mirrored so that x[n-1-i] = -x[i] */
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    double pn, dpn;
    for (int it = 0; it < 100; ++it) {
      legendre_pn(n, z, &pn, &dpn);
      double dz = pn / dpn;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    legendre_pn(n, z, &pn, &dpn);
    double wi = 2.0 / ((1.0 - z * z) * dpn * dpn);
    x[i] = -z; x[n - 1 - i] = z;
    w[i] = wi; w[n - 1 - i] = wi;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

/* Interior rules (weights normalised to sum 1 = quadrature of (1/|T0|) Int).
 * Quadrilateral: tensor Gauss-Legendre.  Triangle: collapsed (Duffy) product
 * rule x = u, y = v (1 - u), weight (1 - u), exact to total degree 2n - 2. */
int orc_interior_rule(int kind, int n, double* xi, double* eta, double* w) {
  double g[16], gw[16];
  if (n < 1 || n > 8) return -1;
  orc_gauss_legendre(n, g, gw);
  int k = 0;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      if (kind == KIND_QUAD) {
        xi[k] = g[a]; eta[k] = g[b]; w[k] = gw[a] * gw[b] / 4.0;
      } else {
        double u = 0.5 * (1.0 + g[a]), v = 0.5 * (1.0 + g[b]);
        xi[k] = u; eta[k] = v * (1.0 - u);
        /* (wa/2)(wb/2)(1-u) integrates over T0 (area 1/2); times 2 -> sum 1 */
        w[k] = 2.0 * (0.5 * gw[a]) * (0.5 * gw[b]) * (1.0 - u);
      }
      ++k;
    }
  return k;
}

/* ------------------------------------------------------------------ */
/* Modal basis (Sec. 1.2: orthonormal Legendre basis, phi^(1) = 1).    */
/* ------------------------------------------------------------------ */
int orc_num_modes(int kind, int deg) {
  (void)kind;
  return (deg + 1) * (deg + 2) / 2;
}

static const int MONO_A[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
static const int MONO_B[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
/* quadrilateral modes as (degree in x, degree in y) */
static const int QUAD_A[10] = {0, 1, 0, 1, 2, 0, 3, 2, 1, 0};
static const int QUAD_B[10] = {0, 0, 1, 1, 0, 2, 0, 1, 2, 3};

/* normalised Legendre polynomial L_n on [-1,1] with (1/2) Int L_n^2 = 1 */
static void leg_norm(int n, double x, double* v, double* d) {
  switch (n) {
    case 0: *v = 1.0; *d = 0.0; break;
    case 1: *v = sqrt(3.0) * x; *d = sqrt(3.0); break;
    case 2: *v = 0.5 * sqrt(5.0) * (3.0 * x * x - 1.0); *d = 3.0 * sqrt(5.0) * x; break;
    default: *v = 0.5 * sqrt(7.0) * (5.0 * x * x * x - 3.0 * x);
             *d = 0.5 * sqrt(7.0) * (15.0 * x * x - 3.0); break;
  }
}

/* (1/|T0|) Int_T0 x^a y^b = 2 a! b! / (a+b+2)! is used below in long double */

/* Gram-Schmidt of the monomials (twice, for round-off) under the exact
 * triangle inner product, carried out in long double because the monomial
 * Gram matrix is ill-conditioned; c[l][j] = coefficient of monomial j in phi_l. */
static long double fact_l(int n) { long double f = 1.0L; for (int i = 2; i <= n; ++i) f *= i; return f; }
static void tri_gram_schmidt(int ML, double c[MAXML][MAXML]) {
  long double G[MAXML][MAXML], cl[MAXML][MAXML];
  for (int j = 0; j < ML; ++j)
    for (int k = 0; k < ML; ++k) {
      int a = MONO_A[j] + MONO_A[k], b = MONO_B[j] + MONO_B[k];
      G[j][k] = 2.0L * fact_l(a) * fact_l(b) / fact_l(a + b + 2);
    }
  for (int l = 0; l < ML; ++l) {
    long double v[MAXML] = {0};
    v[l] = 1.0L;
    for (int pass = 0; pass < 2; ++pass) {
      for (int m = 0; m < l; ++m) {
        long double ip = 0.0L;
        for (int j = 0; j < ML; ++j)
          for (int k = 0; k < ML; ++k) ip += v[j] * G[j][k] * cl[m][k];
        for (int j = 0; j < ML; ++j) v[j] -= ip * cl[m][j];
      }
    }
    long double nn = 0.0L;
    for (int j = 0; j < ML; ++j)
      for (int k = 0; k < ML; ++k) nn += v[j] * G[j][k] * v[k];
    nn = sqrtl(nn);
    for (int j = 0; j < ML; ++j) cl[l][j] = v[j] / nn;
  }
  memset(c, 0, sizeof(double) * MAXML * MAXML);
  for (int l = 0; l < ML; ++l)
    for (int j = 0; j < ML; ++j) c[l][j] = (double)cl[l][j];
}

int orc_basis_eval(int kind, int deg, int npts, const double* xi, const double* eta,
                   double* phi, double* dxi, double* deta) {
  int ML = orc_num_modes(kind, deg);
  if (deg < 1 || deg > 3) return -1;
  double c[MAXML][MAXML];
  if (kind == KIND_TRI) tri_gram_schmidt(ML, c);
  for (int p = 0; p < npts; ++p) {
    double x = xi[p], y = eta[p];
    for (int l = 0; l < ML; ++l) {
      double v, dx, dy;
      if (kind == KIND_QUAD) {
        double lx, dlx, ly, dly;
        leg_norm(QUAD_A[l], x, &lx, &dlx);
        leg_norm(QUAD_B[l], y, &ly, &dly);
        v = lx * ly; dx = dlx * ly; dy = lx * dly;
      } else {
        v = dx = dy = 0.0;
        for (int j = 0; j < ML; ++j) {
          int a = MONO_A[j], b = MONO_B[j];
          double m = pow(x, a) * pow(y, b);
          double mx = a ? a * pow(x, a - 1) * pow(y, b) : 0.0;
          double my = b ? b * pow(x, a) * pow(y, b - 1) : 0.0;
          v += c[l][j] * m; dx += c[l][j] * mx; dy += c[l][j] * my;
        }
      }
      phi[p * ML + l] = v;
      if (dxi) dxi[p * ML + l] = dx;
      if (deta) deta[p * ML + l] = dy;
    }
  }
  return ML;
}

/* ------------------------------------------------------------------ */
/* Euler equations (Eqs. 1-2) and flux derivatives (Sec. 2.2).         */
/* q = (rho, m, n, E), u = m/rho, v = n/rho, p = (g-1)(E - (m^2+n^2)/(2 rho)) */
/* ------------------------------------------------------------------ */
static double pressure(double g, const double* q) {
  return (g - 1.0) * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / q[0]);
}

void orc_flux(double g, const double* q, double* F, double* G) {
  double r = q[0], m = q[1], n = q[2], E = q[3];
  double u = m / r, v = n / r, p = pressure(g, q);
  F[0] = m; F[1] = m * u + p; F[2] = m * v; F[3] = (E + p) * u;
  G[0] = n; G[1] = n * u;     G[2] = n * v + p; G[3] = (E + p) * v;
}

/* First directional derivative d/de F(q + e w) at e = 0 (= F'(q) w, the
 * Jacobian-vector product of Eq. fluxderivs-a).  Derived term by term:
 *   u' = (a - u r)/rho,  v' = (b - v r)/rho,
 *   K' = u a + v b - (u^2+v^2) r / 2   (K = kinetic energy),
 *   p' = (g-1)(e - K'). */
void orc_flux_d1(double g, const double* q, const double* w, double* F1, double* G1) {
  double rho = q[0], m = q[1], n = q[2], E = q[3];
  double r = w[0], a = w[1], b = w[2], e = w[3];
  double u = m / rho, v = n / rho, p = pressure(g, q);
  double du = (a - u * r) / rho, dv = (b - v * r) / rho;
  double dK = u * a + v * b - 0.5 * (u * u + v * v) * r;
  double dp = (g - 1.0) * (e - dK);
  F1[0] = a;
  F1[1] = a * u + m * du + dp;
  F1[2] = a * v + m * dv;
  F1[3] = (e + dp) * u + (E + p) * du;
  G1[0] = b;
  G1[1] = b * u + n * du;
  G1[2] = b * v + n * dv + dp;
  G1[3] = (e + dp) * v + (E + p) * dv;
}

/* Second directional derivative d^2/de^2 F(q + e w) at e = 0
 * (= F''(q)(w,w), the Hessian-vector product of Eq. fluxderivs-b):
 *   u'' = -2 u' r / rho,  v'' = -2 v' r / rho,
 *   K'' = rho (u'^2 + v'^2),  p'' = -(g-1) K''. */
void orc_flux_d2(double g, const double* q, const double* w, double* F2, double* G2) {
  double rho = q[0], m = q[1], n = q[2], E = q[3];
  double r = w[0], a = w[1], b = w[2], e = w[3];
  double u = m / rho, v = n / rho, p = pressure(g, q);
  double du = (a - u * r) / rho, dv = (b - v * r) / rho;
  double ddu = -2.0 * du * r / rho, ddv = -2.0 * dv * r / rho;
  double dK = u * a + v * b - 0.5 * (u * u + v * v) * r;
  double dp = (g - 1.0) * (e - dK);
  double ddp = -(g - 1.0) * rho * (du * du + dv * dv);
  F2[0] = 0.0;
  F2[1] = 2.0 * a * du + m * ddu + ddp;
  F2[2] = 2.0 * a * dv + m * ddv;
  F2[3] = ddp * u + 2.0 * (e + dp) * du + (E + p) * ddu;
  G2[0] = 0.0;
  G2[1] = 2.0 * b * du + n * ddu;
  G2[2] = 2.0 * b * dv + n * ddv + ddp;
  G2[3] = ddp * v + 2.0 * (e + dp) * dv + (E + p) * ddv;
}

/* Third directional derivative d^3/de^3 F(q + e w) at e = 0 (the third
 * derivative of the flux along w, a term of the fourth-order time average).
 * Every quantity along q + e w is kept as its Taylor coefficients in e: rho,
 * m, n, E are linear; rho u = m gives u_k = (m_k - w_rho u_{k-1}) / rho
 * (likewise v); K = (m u + n v)/2 and p = (g-1)(E - K) follow by series
 * products; each flux component is a product of such series, and its third
 * derivative is 3! times the coefficient of e^3. */
static double ser_prod(const double* A, const double* B, int k) {
  double a = 0.0;
  for (int i = 0; i <= k; ++i) a += A[i] * B[k - i];
  return a;
}
void orc_flux_d3(double g, const double* q, const double* w, double* F3, double* G3) {
  double M[4] = {q[1], w[1], 0.0, 0.0}, Nn[4] = {q[2], w[2], 0.0, 0.0}, En[4] = {q[3], w[3], 0.0, 0.0};
  double u[4], v[4], p[4], H[4];
  for (int k = 0; k < 4; ++k) {
    u[k] = (M[k] - (k > 0 ? w[0] * u[k - 1] : 0.0)) / q[0];
    v[k] = (Nn[k] - (k > 0 ? w[0] * v[k - 1] : 0.0)) / q[0];
  }
  for (int k = 0; k < 4; ++k) {
    double K = 0.5 * (ser_prod(M, u, k) + ser_prod(Nn, v, k));
    p[k] = (g - 1.0) * (En[k] - K);
    H[k] = En[k] + p[k];
  }
  F3[0] = 0.0;
  F3[1] = 6.0 * (ser_prod(M, u, 3) + p[3]);
  F3[2] = 6.0 * ser_prod(M, v, 3);
  F3[3] = 6.0 * ser_prod(H, u, 3);
  G3[0] = 0.0;
  G3[1] = 6.0 * ser_prod(Nn, u, 3);
  G3[2] = 6.0 * (ser_prod(Nn, v, 3) + p[3]);
  G3[3] = 6.0 * ser_prod(H, v, 3);
}

/* Mixed second derivative of the flux in the directions a and b, from the
 * second directional derivative by polarisation:
 * (d2 along a+b  -  d2 along a-b) / 4. */
void orc_flux_d11(double g, const double* q, const double* a, const double* b, double* F2, double* G2) {
  double s[4], d[4], Fs[4], Gs[4], Fd[4], Gd[4];
  for (int v = 0; v < NV; ++v) { s[v] = a[v] + b[v]; d[v] = a[v] - b[v]; }
  orc_flux_d2(g, q, s, Fs, Gs);
  orc_flux_d2(g, q, d, Fd, Gd);
  for (int v = 0; v < NV; ++v) { F2[v] = 0.25 * (Fs[v] - Fd[v]); G2[v] = 0.25 * (Gs[v] - Gd[v]); }
}

static double wave_speed_point(double g, const double* q) {
  double u = q[1] / q[0], v = q[2] / q[0];
  double p = pressure(g, q);
  if (p < 0.0) p = 0.0;
  return sqrt(u * u + v * v) + sqrt(g * p / q[0]);
}

/* ------------------------------------------------------------------ */
/* Meshes (Sec. 1.2; edge quantities n_e, e_ik, eps_ik, i_e, j_e of    */
/* Sec. 3.3).  Every element is an affine image x = o + J xi of the    */
/* reference element (square [-1,1]^2 or triangle T0).                 */
/* ------------------------------------------------------------------ */
struct orc_mesh {
  int kind, N, E, nedges;
  double* o;      /* [N][2] */
  double* J;      /* [N][4] row-major: x = o + J xi */
  double* Ji;     /* [N][4] inverse: (dxi/dx, dxi/dy, deta/dx, deta/dy) */
  double* area;   /* [N] */
  double* perim;  /* [N] */
  double* vx;     /* [N][E][2] physical vertices */
  double* nrm;    /* [N][E][2] outward normal scaled by the edge length */
  int* nbr;       /* [N][E] neighbour element or -1 */
  int* nbk;       /* [N][E] neighbour's local edge */
  int* bc;        /* [N][E] boundary code when nbr < 0 */
  int* edge_of;   /* [N][E] edge id */
  int* eps;       /* [N][E] +1 if the edge normal points out of this element */
  int* e_i; int* e_ki; int* e_j; int* e_kj; /* edges: owner i_e (normal outward), j_e */
  double hmin;    /* min_i 2|T_i|/P_i */
  double hdx;     /* characteristic spacing per element, stored in sdx */
  double* sdx;    /* [N] dx used by the shock limiter */
};

static const double QREF[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
static const double TREF[3][2] = {{0, 0}, {1, 0}, {0, 1}};

static orc_mesh* mesh_alloc(int kind, int N) {
  orc_mesh* m = (orc_mesh*)calloc(1, sizeof(orc_mesh));
  m->kind = kind; m->N = N; m->E = kind == KIND_QUAD ? 4 : 3;
  int E = m->E;
  m->o = calloc((size_t)N * 2, sizeof(double));
  m->J = calloc((size_t)N * 4, sizeof(double));
  m->Ji = calloc((size_t)N * 4, sizeof(double));
  m->area = calloc((size_t)N, sizeof(double));
  m->perim = calloc((size_t)N, sizeof(double));
  m->sdx = calloc((size_t)N, sizeof(double));
  m->vx = calloc((size_t)N * E * 2, sizeof(double));
  m->nrm = calloc((size_t)N * E * 2, sizeof(double));
  m->nbr = calloc((size_t)N * E, sizeof(int));
  m->nbk = calloc((size_t)N * E, sizeof(int));
  m->bc = calloc((size_t)N * E, sizeof(int));
  m->edge_of = calloc((size_t)N * E, sizeof(int));
  m->eps = calloc((size_t)N * E, sizeof(int));
  return m;
}

/* geometry from the physical vertices: affine map, area, normals */
static void mesh_geometry(orc_mesh* m) {
  int E = m->E;
  double T0 = m->kind == KIND_QUAD ? 4.0 : 0.5;
  m->hmin = 1e300;
  for (int i = 0; i < m->N; ++i) {
    double* v = m->vx + (size_t)i * E * 2;
    double *o = m->o + 2 * i, *J = m->J + 4 * i, *Ji = m->Ji + 4 * i;
    if (m->kind == KIND_QUAD) {
      o[0] = 0.5 * (v[0] + v[2]); o[1] = 0.5 * (v[1] + v[5]);
      J[0] = 0.5 * (v[2] - v[0]); J[1] = 0.0; J[2] = 0.0; J[3] = 0.5 * (v[5] - v[1]);
    } else {
      o[0] = v[0]; o[1] = v[1];
      J[0] = v[2] - v[0]; J[1] = v[4] - v[0]; J[2] = v[3] - v[1]; J[3] = v[5] - v[1];
    }
    double det = J[0] * J[3] - J[1] * J[2];
    Ji[0] = J[3] / det; Ji[1] = -J[1] / det; Ji[2] = -J[2] / det; Ji[3] = J[0] / det;
    m->area[i] = T0 * det;
    double P = 0.0;
    for (int k = 0; k < E; ++k) {
      int k1 = (k + 1) % E;
      double xa = v[2 * k], ya = v[2 * k + 1], xb = v[2 * k1], yb = v[2 * k1 + 1];
      double* n = m->nrm + ((size_t)i * E + k) * 2;
      n[0] = yb - ya; n[1] = -(xb - xa);
      P += sqrt(n[0] * n[0] + n[1] * n[1]);
    }
    m->perim[i] = P;
    double h = 2.0 * m->area[i] / P;
    if (h < m->hmin) m->hmin = h;
    m->sdx[i] = m->kind == KIND_QUAD ? 2.0 * J[0] : sqrt(2.0 * m->area[i]);
  }
}

/* edge list: owner i_e is the element whose outward normal is n_e */
static void mesh_edges(orc_mesh* m) {
  int E = m->E, N = m->N;
  m->e_i = malloc(sizeof(int) * (size_t)N * E);
  m->e_ki = malloc(sizeof(int) * (size_t)N * E);
  m->e_j = malloc(sizeof(int) * (size_t)N * E);
  m->e_kj = malloc(sizeof(int) * (size_t)N * E);
  for (int i = 0; i < N * E; ++i) m->edge_of[i] = -1;
  int ne = 0;
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < E; ++k) {
      if (m->edge_of[i * E + k] >= 0) continue;
      int j = m->nbr[i * E + k], kj = m->nbk[i * E + k];
      m->e_i[ne] = i; m->e_ki[ne] = k; m->e_j[ne] = j; m->e_kj[ne] = kj;
      m->edge_of[i * E + k] = ne; m->eps[i * E + k] = 1;
      if (j >= 0) { m->edge_of[j * E + kj] = ne; m->eps[j * E + kj] = -1; }
      ++ne;
    }
  m->nedges = ne;
}

/* nx*ny axis-aligned cells; with a mask, the cells with mask[iy*nx+ix] == 0
 * are left out (elements numbered in row order of the cells kept) and the
 * faces a kept cell shares with a left-out one get the code mask_bc. */
orc_mesh* orc_mesh_cartesian_masked(int nx, int ny, double x0, double x1, double y0, double y1, const int* bc,
                                    const unsigned char* mask, int mask_bc) {
  if (nx < 1 || ny < 1) return NULL;
  if ((bc[0] == BC_PERIODIC) != (bc[1] == BC_PERIODIC)) return NULL;
  if ((bc[2] == BC_PERIODIC) != (bc[3] == BC_PERIODIC)) return NULL;
  int* id = malloc(sizeof(int) * (size_t)nx * ny);
  int N = 0;
  for (int c = 0; c < nx * ny; ++c) id[c] = (!mask || mask[c]) ? N++ : -1;
  if (N < 1) { free(id); return NULL; }
  orc_mesh* m = mesh_alloc(KIND_QUAD, N);
  double* X = malloc(sizeof(double) * (nx + 1));
  double* Y = malloc(sizeof(double) * (ny + 1));
  for (int i = 0; i <= nx; ++i) X[i] = x0 + (x1 - x0) * i / nx;
  for (int j = 0; j <= ny; ++j) Y[j] = y0 + (y1 - y0) * j / ny;
  for (int iy = 0; iy < ny; ++iy)
    for (int ix = 0; ix < nx; ++ix) {
      int c = iy * nx + ix, i = id[c];
      if (i < 0) continue;
      double* v = m->vx + (size_t)i * 8;
      v[0] = X[ix]; v[1] = Y[iy]; v[2] = X[ix + 1]; v[3] = Y[iy];
      v[4] = X[ix + 1]; v[5] = Y[iy + 1]; v[6] = X[ix]; v[7] = Y[iy + 1];
      /* local edges: 0 bottom, 1 right, 2 top, 3 left (counter-clockwise) */
      int nb[4], nk[4] = {2, 3, 0, 1}, bcode[4] = {bc[2], bc[1], bc[3], bc[0]};
      nb[0] = iy > 0 ? c - nx : (bc[2] == BC_PERIODIC ? (ny - 1) * nx + ix : -1);
      nb[1] = ix < nx - 1 ? c + 1 : (bc[1] == BC_PERIODIC ? iy * nx : -1);
      nb[2] = iy < ny - 1 ? c + nx : (bc[3] == BC_PERIODIC ? ix : -1);
      nb[3] = ix > 0 ? c - 1 : (bc[0] == BC_PERIODIC ? iy * nx + nx - 1 : -1);
      for (int k = 0; k < 4; ++k) {
        int j = nb[k] >= 0 ? id[nb[k]] : -1;
        m->nbr[i * 4 + k] = j;
        m->nbk[i * 4 + k] = j >= 0 ? nk[k] : -1;
        m->bc[i * 4 + k] = j >= 0 ? BC_PERIODIC : (nb[k] >= 0 ? mask_bc : bcode[k]);
      }
    }
  free(X); free(Y); free(id);
  mesh_geometry(m);
  mesh_edges(m);
  return m;
}

orc_mesh* orc_mesh_cartesian(int nx, int ny, double x0, double x1, double y0, double y1, const int* bc) {
  return orc_mesh_cartesian_masked(nx, ny, x0, x1, y0, y1, bc, NULL, BC_REFLECT);
}

typedef struct { int a, b, elem, k; } half_edge;
static int cmp_half(const void* x, const void* y) {
  const half_edge *p = x, *q = y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  if (p->elem != q->elem) return p->elem < q->elem ? -1 : 1;
  return p->k - q->k;
}

orc_mesh* orc_mesh_triangles(int nv, const double* xy, int nt, const int* tv, const int* ebc) {
  if (nt < 1) return NULL;
  orc_mesh* m = mesh_alloc(KIND_TRI, nt);
  half_edge* h = malloc(sizeof(half_edge) * (size_t)nt * 3);
  for (int i = 0; i < nt; ++i) {
    for (int k = 0; k < 3; ++k) {
      int vi = tv[3 * i + k];
      if (vi < 0 || vi >= nv) { free(h); orc_mesh_free(m); return NULL; }
      m->vx[(size_t)i * 6 + 2 * k] = xy[2 * vi];
      m->vx[(size_t)i * 6 + 2 * k + 1] = xy[2 * vi + 1];
      int va = tv[3 * i + k], vb = tv[3 * i + (k + 1) % 3];
      h[3 * i + k].a = va < vb ? va : vb;
      h[3 * i + k].b = va < vb ? vb : va;
      h[3 * i + k].elem = i; h[3 * i + k].k = k;
      m->nbr[3 * i + k] = -1; m->nbk[3 * i + k] = -1;
      m->bc[3 * i + k] = ebc ? ebc[3 * i + k] : BC_TRANSPARENT;
    }
  }
  qsort(h, (size_t)nt * 3, sizeof(half_edge), cmp_half);
  for (int s = 0; s + 1 < nt * 3; ++s) {
    if (h[s].a == h[s + 1].a && h[s].b == h[s + 1].b) {
      int i = h[s].elem, k = h[s].k, j = h[s + 1].elem, kj = h[s + 1].k;
      m->nbr[3 * i + k] = j; m->nbk[3 * i + k] = kj;
      m->nbr[3 * j + kj] = i; m->nbk[3 * j + kj] = k;
      m->bc[3 * i + k] = BC_PERIODIC; m->bc[3 * j + kj] = BC_PERIODIC;
      ++s;
    }
  }
  free(h);
  mesh_geometry(m);
  for (int i = 0; i < nt; ++i)
    if (m->area[i] <= 0.0) { orc_mesh_free(m); return NULL; }
  mesh_edges(m);
  return m;
}

void orc_mesh_free(orc_mesh* m) {
  if (!m) return;
  free(m->o); free(m->J); free(m->Ji); free(m->area); free(m->perim); free(m->sdx);
  free(m->vx); free(m->nrm); free(m->nbr); free(m->nbk); free(m->bc); free(m->edge_of);
  free(m->eps); free(m->e_i); free(m->e_ki); free(m->e_j); free(m->e_kj);
  free(m);
}
int orc_mesh_num_elements(const orc_mesh* m) { return m->N; }
int orc_mesh_num_edges(const orc_mesh* m) { return m->nedges; }
int orc_mesh_edges_per_element(const orc_mesh* m) { return m->E; }
void orc_mesh_geometry(const orc_mesh* m, double* area, double* perim, double* cx, double* cy) {
  for (int i = 0; i < m->N; ++i) {
    if (area) area[i] = m->area[i];
    if (perim) perim[i] = m->perim[i];
    double sx = 0, sy = 0;
    for (int k = 0; k < m->E; ++k) { sx += m->vx[(size_t)i * m->E * 2 + 2 * k];
                                     sy += m->vx[(size_t)i * m->E * 2 + 2 * k + 1]; }
    if (cx) cx[i] = sx / m->E;
    if (cy) cy[i] = sy / m->E;
  }
}

/* ------------------------------------------------------------------ */
/* Solver tables                                                       */
/* ------------------------------------------------------------------ */
struct orc_solver {
  const orc_mesh* m;
  int deg, ML, E, NQ, MQ, NPT, NPJ;
  double gamma, eps0, alpha0;
  int shock_limiter;
  int moment_exact;                         /* Step 2 by the exact root instead of the secant */
  int llf_global;                           /* Eq. LLF point flux with the global s instead of the local speed */
  int ck_order;                             /* 3 (Eq. taylor3-flux) or 4 (one more term of the series) */
  double qx[MAXQ], qy[MAXQ], qw[MAXQ];
  double gs[MAXMQ], gw[MAXMQ];
  /* points: 0..NQ-1 interior, then edge k point p at NQ + k*MQ + p */
  double px[MAXPTS], py[MAXPTS];
  double phi[MAXPTS][MAXML], dxi[MAXPTS][MAXML], deta[MAXPTS][MAXML];
  double jx[MAXPJ], jy[MAXPJ], jw[MAXPJ], jphi[MAXPJ][MAXML];
  /* per-step work arrays */
  double *V, *tq, *tqt, *tqtt, *tqttt, *tF, *tG;   /* V[N][ML][4]; traces [N][E][MQ][4] */
  double *fstar, *flxw, *flxf;              /* per edge: [ne][MQ][4], [ne][4], [ne][4] */
  double *prop;                             /* [N][E] Lambda proposals */
  double last_dt;
  double qinf[4];                           /* conserved state of inflow boundaries */
};

orc_solver* orc_solver_new(const orc_mesh* m, int deg, double gamma) {
  if (deg < 1 || deg > 3) return NULL;
  orc_solver* s = calloc(1, sizeof(orc_solver));
  s->m = m; s->deg = deg; s->E = m->E; s->gamma = gamma;
  s->eps0 = 1e-12; s->alpha0 = 500.0; s->shock_limiter = 1; s->ck_order = 3;
  s->ML = orc_num_modes(m->kind, deg);
  int n = deg + 1;
  s->NQ = orc_interior_rule(m->kind, n, s->qx, s->qy, s->qw);
  s->MQ = n;
  orc_gauss_legendre(n, s->gs, s->gw);
  for (int k = 0; k < s->NQ; ++k) { s->px[k] = s->qx[k]; s->py[k] = s->qy[k]; }
  const double(*ref)[2] = m->kind == KIND_QUAD ? QREF : TREF;
  for (int k = 0; k < s->E; ++k) {
    int k1 = (k + 1) % s->E;
    for (int p = 0; p < s->MQ; ++p) {
      double t = 0.5 * (s->gs[p] + 1.0);
      int idx = s->NQ + k * s->MQ + p;
      s->px[idx] = ref[k][0] + t * (ref[k1][0] - ref[k][0]);
      s->py[idx] = ref[k][1] + t * (ref[k1][1] - ref[k][1]);
    }
  }
  s->NPT = s->NQ + s->E * s->MQ;
  double ph[MAXPTS * MAXML], dx[MAXPTS * MAXML], dy[MAXPTS * MAXML];
  orc_basis_eval(m->kind, deg, s->NPT, s->px, s->py, ph, dx, dy);
  for (int p = 0; p < s->NPT; ++p)
    for (int l = 0; l < s->ML; ++l) {
      s->phi[p][l] = ph[p * s->ML + l];
      s->dxi[p][l] = dx[p * s->ML + l];
      s->deta[p][l] = dy[p * s->ML + l];
    }
  /* projection rule: deg + 3 points per direction */
  s->NPJ = orc_interior_rule(m->kind, deg + 3, s->jx, s->jy, s->jw);
  orc_basis_eval(m->kind, deg, s->NPJ, s->jx, s->jy, ph, NULL, NULL);
  for (int p = 0; p < s->NPJ; ++p)
    for (int l = 0; l < s->ML; ++l) s->jphi[p][l] = ph[p * s->ML + l];
  size_t N = (size_t)m->N, E = (size_t)m->E, MQ = (size_t)s->MQ, ne = (size_t)m->nedges;
  s->V = malloc(sizeof(double) * N * s->ML * NV);
  s->tq = malloc(sizeof(double) * N * E * MQ * NV);
  s->tqt = malloc(sizeof(double) * N * E * MQ * NV);
  s->tqtt = malloc(sizeof(double) * N * E * MQ * NV);
  s->tqttt = malloc(sizeof(double) * N * E * MQ * NV);
  s->tF = malloc(sizeof(double) * N * E * MQ * NV);
  s->tG = malloc(sizeof(double) * N * E * MQ * NV);
  s->fstar = malloc(sizeof(double) * ne * MQ * NV);
  s->flxw = malloc(sizeof(double) * ne * NV);
  s->flxf = malloc(sizeof(double) * ne * NV);
  s->prop = malloc(sizeof(double) * N * E);
  return s;
}

void orc_solver_free(orc_solver* s) {
  if (!s) return;
  free(s->V); free(s->tq); free(s->tqt); free(s->tqtt); free(s->tqttt); free(s->tF); free(s->tG);
  free(s->fstar); free(s->flxw); free(s->flxf); free(s->prop);
  free(s);
}
void orc_solver_set_params(orc_solver* s, double eps0, double alpha0, int shock_limiter) {
  s->eps0 = eps0; s->alpha0 = alpha0; s->shock_limiter = shock_limiter;
}

/* Sec. 3.1 notes that the optimal theta could be computed exactly instead
 * of by Lemma 1's secant; flag 1 selects that variant. */
void orc_solver_set_moment_exact(orc_solver* s, int flag) { s->moment_exact = flag; }

/* Eq. LLF names the dissipation speed of the high-order point flux "an
 * estimate of the maximum global wave speed"; flag 1 uses the global s there
 * (the literal reading), flag 0 (default) the local Lax-Friedrichs speed of
 * the two traces (see the readings at the top of this file). */
void orc_solver_set_llf_global(orc_solver* s, int flag) { s->llf_global = flag; }

/* Order in time of the CK flux: 3 is Eq. taylor3-flux (F + dt/2 F_t +
 * dt^2/6 F_tt); 4 adds dt^3/24 F_ttt, the next term of the same series, for
 * P3 elements (the higher-order direction the conclusions name).  Returns 1
 * for an order other than 3 or 4. */
int orc_solver_set_ck_order(orc_solver* s, int order) {
  if (order != 3 && order != 4) return 1;
  s->ck_order = order;
  return 0;
}

/* the state of inflow boundaries from primitive values (rho, u, v, p) */
void orc_solver_set_inflow(orc_solver* s, const double* prim) {
  s->qinf[0] = prim[0];
  s->qinf[1] = prim[0] * prim[1];
  s->qinf[2] = prim[0] * prim[2];
  s->qinf[3] = prim[3] / (s->gamma - 1.0) + 0.5 * prim[0] * (prim[1] * prim[1] + prim[2] * prim[2]);
}
int orc_solver_num_modes(const orc_solver* s) { return s->ML; }
int orc_solver_num_points(const orc_solver* s) { return s->NPT; }
int orc_projection_num_points(const orc_solver* s) { return s->NPJ; }

void orc_projection_points(const orc_solver* s, double* xy) {
  const orc_mesh* m = s->m;
  for (int i = 0; i < m->N; ++i) {
    const double *o = m->o + 2 * i, *J = m->J + 4 * i;
    for (int p = 0; p < s->NPJ; ++p) {
      double* r = xy + ((size_t)i * s->NPJ + p) * 2;
      r[0] = o[0] + J[0] * s->jx[p] + J[1] * s->jy[p];
      r[1] = o[1] + J[2] * s->jx[p] + J[3] * s->jy[p];
    }
  }
}
void orc_projection_weights(const orc_solver* s, double* w) {
  for (int p = 0; p < s->NPJ; ++p) w[p] = s->jw[p];
}

/* L2 projection of the initial condition (Sec. 1.2; Q^(l) = (1/|T0|) Int q phi_l)
 * from primitive values (rho, u, v, p) at the projection points; the
 * energy follows Eq. eos. */
void orc_project(const orc_solver* s, const double* prim, double* Q) {
  int ML = s->ML;
  for (int i = 0; i < s->m->N; ++i) {
    double* Qi = Q + (size_t)i * NV * ML;
    for (int c = 0; c < NV * ML; ++c) Qi[c] = 0.0;
    for (int p = 0; p < s->NPJ; ++p) {
      const double* w = prim + ((size_t)i * s->NPJ + p) * 4;
      double q[4] = {w[0], w[0] * w[1], w[0] * w[2],
                     w[3] / (s->gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2])};
      for (int v = 0; v < NV; ++v)
        for (int l = 0; l < ML; ++l) Qi[v * ML + l] += s->jw[p] * q[v] * s->jphi[p][l];
    }
  }
}

static void eval_point(const orc_solver* s, const double* Qi, const double* phi, double* q) {
  for (int v = 0; v < NV; ++v) {
    double a = 0.0;
    for (int l = 0; l < s->ML; ++l) a += Qi[v * s->ML + l] * phi[l];
    q[v] = a;
  }
}

void orc_eval_projection_points(const orc_solver* s, const double* Q, double* q) {
  for (int i = 0; i < s->m->N; ++i)
    for (int p = 0; p < s->NPJ; ++p)
      eval_point(s, Q + (size_t)i * NV * s->ML, s->jphi[p], q + ((size_t)i * s->NPJ + p) * 4);
}
void orc_limiter_points(const orc_solver* s, double* xy) {
  const orc_mesh* m = s->m;
  for (int i = 0; i < m->N; ++i) {
    const double *o = m->o + 2 * i, *J = m->J + 4 * i;
    for (int p = 0; p < s->NPT; ++p) {
      double* r = xy + ((size_t)i * s->NPT + p) * 2;
      r[0] = o[0] + J[0] * s->px[p] + J[1] * s->py[p];
      r[1] = o[1] + J[2] * s->px[p] + J[3] * s->py[p];
    }
  }
}

double orc_last_fluxes(const orc_solver* s, double* fw, double* ff) {
  const orc_mesh* m = s->m;
  for (int i = 0; i < m->N; ++i)
    for (int k = 0; k < m->E; ++k) {
      int e = m->edge_of[i * m->E + k];
      double ek = m->eps[i * m->E + k];
      for (int v = 0; v < NV; ++v) {
        fw[((size_t)i * m->E + k) * NV + v] = ek * s->flxw[(size_t)e * NV + v];
        ff[((size_t)i * m->E + k) * NV + v] = ek * s->flxf[(size_t)e * NV + v];
      }
    }
  return s->last_dt;
}

void orc_eval_limiter_points(const orc_solver* s, const double* Q, double* q) {
  for (int i = 0; i < s->m->N; ++i)
    for (int p = 0; p < s->NPT; ++p)
      eval_point(s, Q + (size_t)i * NV * s->ML, s->phi[p], q + ((size_t)i * s->NPT + p) * 4);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.1: moment limiter (Steps 0-2) on one element.                */
/* ------------------------------------------------------------------ */
static double moment_limit_element(const orc_solver* s, double* Qi, int* status) {
  int ML = s->ML;
  double g = s->gamma;
  double qbar[4] = {Qi[0], Qi[ML], Qi[2 * ML], Qi[3 * ML]};
  /* Step 0: positivity of the averages is assumed; if violated, flatten */
  double pbar = qbar[0] > 0.0 ? pressure(g, qbar) : -1.0;
  if (!(qbar[0] > 0.0) || !(pbar > 0.0)) {
    *status |= ORC_ST_NONPOSITIVE;
    for (int v = 0; v < NV; ++v)
      for (int l = 1; l < ML; ++l) Qi[v * ML + l] = 0.0;
    return 0.0;
  }
  /* deviations q~_m from the average at every limiter point */
  double dev[MAXPTS][4];
  for (int p = 0; p < s->NPT; ++p)
    for (int v = 0; v < NV; ++v) {
      double a = 0.0;
      for (int l = 1; l < ML; ++l) a += Qi[v * ML + l] * s->phi[p][l];
      dev[p][v] = a;
    }
  /* Step 1 (Eq. rho-theta): largest theta_rho with rho_m >= eps */
  double eps_r = fmin(s->eps0, 0.5 * qbar[0]);
  double th_r = 1.0;
  for (int p = 0; p < s->NPT; ++p) {
    double rm = qbar[0] + dev[p][0];
    if (rm < eps_r) {
      double t = (qbar[0] - eps_r) / (qbar[0] - rm);
      if (t < th_r) th_r = t;
    }
  }
  /* Step 2 (Lemma 1): secant through (0, p0) and (theta_rho, p^{theta_rho}_m);
   * or, with moment_exact, the point's exact crossing of eps_p */
  double eps_p = fmin(s->eps0, 0.5 * pbar);
  double th = th_r;
  for (int p = 0; p < s->NPT; ++p) {
    double qt[4];
    for (int v = 0; v < NV; ++v) qt[v] = qbar[v] + th_r * dev[p][v];
    double pt = pressure(g, qt);
    if (pt < eps_p) {
      double t;
      if (s->moment_exact) {
        /* (rho p)^theta - eps_p rho^theta over (g-1) along q(theta) = qbar + theta dev
         * (the quadratic of Eq. product-rho-p shifted by the floor): h0 + h1 t + h2 t^2,
         * positive at 0, negative at theta_rho: its one root there, cancellation-free */
        double kappa = eps_p / (g - 1.0);
        const double* d = dev[p];
        double h0 = qbar[0] * qbar[3] - 0.5 * (qbar[1] * qbar[1] + qbar[2] * qbar[2]) - kappa * qbar[0];
        double h1 = qbar[0] * d[3] + d[0] * qbar[3] - (qbar[1] * d[1] + qbar[2] * d[2]) - kappa * d[0];
        double h2 = d[0] * d[3] - 0.5 * (d[1] * d[1] + d[2] * d[2]);
        double disc = h1 * h1 - 4.0 * h0 * h2;
        if (disc < 0.0) disc = 0.0;
        double den = -h1 + sqrt(disc);
        t = den > 0.0 ? 2.0 * h0 / den : 0.0;
        if (t > th_r) t = th_r;
      } else {
        t = th_r * (pbar - eps_p) / (pbar - pt);
      }
      if (t < th) th = t;
    }
  }
  if (th < 0.0) th = 0.0;
  if (th < 1.0)
    for (int v = 0; v < NV; ++v)
      for (int l = 1; l < ML; ++l) Qi[v * ML + l] *= th;
  return th;
}

double orc_moment_limit(const orc_solver* s, double* Q, double* theta, int* status) {
  int st = 0;
  double mn = 1.0;
#pragma omp parallel for reduction(| : st) reduction(min : mn) schedule(static)
  for (int i = 0; i < s->m->N; ++i) {
    int sti = 0;
    double t = moment_limit_element(s, Q + (size_t)i * NV * s->ML, &sti);
    if (theta) theta[i] = t;
    st |= sti;
    if (t < mn) mn = t;
  }
  if (status) *status |= st;
  return mn;
}

/* Global wave speed s (Eq. LLF; read as the maximum of |u| + c over the
 * cell averages and the limited point values). */
double orc_wave_speed(const orc_solver* s, const double* Q) {
  double smax = 0.0;
#pragma omp parallel for reduction(max : smax) schedule(static)
  for (int i = 0; i < s->m->N; ++i) {
    const double* Qi = Q + (size_t)i * NV * s->ML;
    double qbar[4] = {Qi[0], Qi[s->ML], Qi[2 * s->ML], Qi[3 * s->ML]};
    double a = wave_speed_point(s->gamma, qbar);
    if (a > smax) smax = a;
    for (int p = 0; p < s->NPT; ++p) {
      double q[4];
      eval_point(s, Qi, s->phi[p], q);
      double b = wave_speed_point(s->gamma, q);
      if (b > smax) smax = b;
    }
  }
  return smax;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2-2.3: Cauchy-Kovalevskaya time-averaged flux on one element */
/* Steps 1-2: project F onto the basis with the interior rule, take    */
/* q_t = -div F^h, F_t = F'(q) q_t, project, q_tt = -div F_t^h,        */
/* F_tt = F''(q)(q_t,q_t) + F'(q) q_tt, F_T = F + dt/2 F_t + dt^2/6 F_tt */
/* (Eq. taylor3-flux).  Step 3: volume integral V^(l) = Int grad phi.F_T. */
/* ------------------------------------------------------------------ */
static void ck_element(const orc_solver* s, const double* Qi, int i, double dt,
                       double (*q)[4], double (*qt)[4], double (*qtt)[4],
                       double (*FT)[4], double (*GT)[4], double (*V)[4], double (*qttt)[4]) {
  const orc_mesh* m = s->m;
  int ML = s->ML, NQ = s->NQ, NPT = s->NPT;
  double g = s->gamma;
  const double* Ji = m->Ji + 4 * i;
  /* physical gradients of the basis at all points */
  double bx[MAXPTS][MAXML], by[MAXPTS][MAXML];
  for (int p = 0; p < NPT; ++p)
    for (int l = 0; l < ML; ++l) {
      bx[p][l] = Ji[0] * s->dxi[p][l] + Ji[2] * s->deta[p][l];
      by[p][l] = Ji[1] * s->dxi[p][l] + Ji[3] * s->deta[p][l];
    }
  double F[MAXPTS][4], G[MAXPTS][4];
  for (int p = 0; p < NPT; ++p) {
    eval_point(s, Qi, s->phi[p], q[p]);
    orc_flux(g, q[p], F[p], G[p]);
  }
  /* Step 1: Galerkin expansion of F and G */
  double Fh[MAXML][4], Gh[MAXML][4];
  for (int l = 0; l < ML; ++l)
    for (int v = 0; v < NV; ++v) {
      double a = 0.0, b = 0.0;
      for (int k = 0; k < NQ; ++k) {
        a += s->qw[k] * F[k][v] * s->phi[k][l];
        b += s->qw[k] * G[k][v] * s->phi[k][l];
      }
      Fh[l][v] = a; Gh[l][v] = b;
    }
  /* q_t = -div F^h and F_t = F'(q) q_t (Eq. fluxderivs-a) */
  double Ft[MAXPTS][4], Gt[MAXPTS][4];
  for (int p = 0; p < NPT; ++p) {
    for (int v = 0; v < NV; ++v) {
      double d = 0.0;
      for (int l = 0; l < ML; ++l) d += Fh[l][v] * bx[p][l] + Gh[l][v] * by[p][l];
      qt[p][v] = -d;
    }
    orc_flux_d1(g, q[p], qt[p], Ft[p], Gt[p]);
  }
  double Fth[MAXML][4], Gth[MAXML][4];
  for (int l = 0; l < ML; ++l)
    for (int v = 0; v < NV; ++v) {
      double a = 0.0, b = 0.0;
      for (int k = 0; k < NQ; ++k) {
        a += s->qw[k] * Ft[k][v] * s->phi[k][l];
        b += s->qw[k] * Gt[k][v] * s->phi[k][l];
      }
      Fth[l][v] = a; Gth[l][v] = b;
    }
  /* q_tt = -div F_t^h and F_tt (Eq. fluxderivs-b) at every point */
  double Ftt[MAXPTS][4], Gtt[MAXPTS][4];
  for (int p = 0; p < NPT; ++p) {
    for (int v = 0; v < NV; ++v) {
      double d = 0.0;
      for (int l = 0; l < ML; ++l) d += Fth[l][v] * bx[p][l] + Gth[l][v] * by[p][l];
      qtt[p][v] = -d;
    }
    double F2[4], G2[4], F1[4], G1[4];
    orc_flux_d2(g, q[p], qt[p], F2, G2);
    orc_flux_d1(g, q[p], qtt[p], F1, G1);
    for (int v = 0; v < NV; ++v) { Ftt[p][v] = F2[v] + F1[v]; Gtt[p][v] = G2[v] + G1[v]; }
  }
  /* F_T = F + dt/2 F_t + dt^2/6 F_tt (Eq. taylor3-flux) */
  for (int p = 0; p < NPT; ++p)
    for (int v = 0; v < NV; ++v) {
      FT[p][v] = F[p][v] + dt / 2.0 * Ft[p][v] + dt * dt / 6.0 * Ftt[p][v];
      GT[p][v] = G[p][v] + dt / 2.0 * Gt[p][v] + dt * dt / 6.0 * Gtt[p][v];
    }
  /* Fourth order in time (the next term of the same Taylor series of the
   * time-averaged flux): q_ttt = -div F_tt^h, F_ttt = F'''(q)(q_t,q_t,q_t)
   * + 3 F''(q)(q_t, q_tt) + F'(q) q_ttt, F_T += dt^3/24 F_ttt */
  for (int p = 0; p < NPT; ++p)
    for (int v = 0; v < NV; ++v) qttt[p][v] = 0.0;
  if (s->ck_order == 4) {
    double Ftth[MAXML][4], Gtth[MAXML][4];
    for (int l = 0; l < ML; ++l)
      for (int v = 0; v < NV; ++v) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < NQ; ++k) {
          a += s->qw[k] * Ftt[k][v] * s->phi[k][l];
          b += s->qw[k] * Gtt[k][v] * s->phi[k][l];
        }
        Ftth[l][v] = a; Gtth[l][v] = b;
      }
    for (int p = 0; p < NPT; ++p) {
      for (int v = 0; v < NV; ++v) {
        double d = 0.0;
        for (int l = 0; l < ML; ++l) d += Ftth[l][v] * bx[p][l] + Gtth[l][v] * by[p][l];
        qttt[p][v] = -d;
      }
      double F3[4], G3[4], Fm[4], Gm[4], F1[4], G1[4];
      orc_flux_d3(g, q[p], qt[p], F3, G3);
      orc_flux_d11(g, q[p], qt[p], qtt[p], Fm, Gm);
      orc_flux_d1(g, q[p], qttt[p], F1, G1);
      for (int v = 0; v < NV; ++v) {
        FT[p][v] += dt * dt * dt / 24.0 * (F3[v] + 3.0 * Fm[v] + F1[v]);
        GT[p][v] += dt * dt * dt / 24.0 * (G3[v] + 3.0 * Gm[v] + G1[v]);
      }
    }
  }
  /* Step 3: interior integral of Eq. EulerStepExactGalerkin */
  for (int l = 0; l < ML; ++l)
    for (int v = 0; v < NV; ++v) {
      double a = 0.0;
      for (int k = 0; k < NQ; ++k) a += s->qw[k] * (bx[k][l] * FT[k][v] + by[k][l] * GT[k][v]);
      V[l][v] = m->area[i] * a;
    }
}

void orc_ck_element(const orc_solver* s, const double* Q, int i, double dt, double* q,
                    double* qt, double* qtt, double* FT, double* GT, double* V) {
  double a[MAXPTS][4], b[MAXPTS][4], c[MAXPTS][4], d[MAXPTS][4], e[MAXPTS][4], f[MAXML][4], h[MAXPTS][4];
  ck_element(s, Q + (size_t)i * NV * s->ML, i, dt, a, b, c, d, e, f, h);
  for (int p = 0; p < s->NPT; ++p)
    for (int v = 0; v < NV; ++v) {
      if (q) q[p * 4 + v] = a[p][v];
      if (qt) qt[p * 4 + v] = b[p][v];
      if (qtt) qtt[p * 4 + v] = c[p][v];
      if (FT) FT[p * 4 + v] = d[p][v];
      if (GT) GT[p * 4 + v] = e[p][v];
    }
  if (V)
    for (int l = 0; l < s->ML; ++l)
      for (int v = 0; v < NV; ++v) V[l * 4 + v] = f[l][v];
}

/* Sec. 2.4: exterior state at a boundary point; the same map is applied to
 * q, q_t and q_tt.  Reflective flips the normal momentum, transparent copies.
 * Inflow (the shock-diffraction problems of Sec. 4) prescribes a steady
 * state: q -> q_inflow, q_t and q_tt -> 0 (deriv = 1 marks those). */
static void boundary_state(int bc, const double* nh, const double* qin, double* qout, const double* qinflow,
                           int deriv) {
  if (bc == BC_INFLOW) {
    for (int v = 0; v < 4; ++v) qout[v] = deriv ? 0.0 : qinflow[v];
    return;
  }
  qout[0] = qin[0]; qout[3] = qin[3];
  double mn = qin[1] * nh[0] + qin[2] * nh[1];
  double mt0 = qin[1] - mn * nh[0], mt1 = qin[2] - mn * nh[1];
  double sgn = bc == BC_REFLECT ? -1.0 : 1.0;
  qout[1] = mt0 + sgn * mn * nh[0];
  qout[2] = mt1 + sgn * mn * nh[1];
}

/* F_T from q, q_t, q_tt at one point (used for boundary states) */
static void ft_from_derivs(double g, double dt, const double* q, const double* qt, const double* qtt,
                           const double* qttt, double* FT, double* GT) {
  double F[4], G[4], F1[4], G1[4], F2[4], G2[4], F3[4], G3[4];
  orc_flux(g, q, F, G);
  orc_flux_d1(g, q, qt, F1, G1);
  orc_flux_d2(g, q, qt, F2, G2);
  orc_flux_d1(g, q, qtt, F3, G3);
  for (int v = 0; v < NV; ++v) {
    FT[v] = F[v] + dt / 2.0 * F1[v] + dt * dt / 6.0 * (F2[v] + F3[v]);
    GT[v] = G[v] + dt / 2.0 * G1[v] + dt * dt / 6.0 * (G2[v] + G3[v]);
  }
  if (qttt) {   /* fourth order: + dt^3/24 (F'''(q_t)^3 + 3 F''(q_t, q_tt) + F'(q_ttt)) */
    double A[4], B[4], C2[4], D2[4], E1[4], G1b[4];
    orc_flux_d3(g, q, qt, A, B);
    orc_flux_d11(g, q, qt, qtt, C2, D2);
    orc_flux_d1(g, q, qttt, E1, G1b);
    for (int v = 0; v < NV; ++v) {
      FT[v] += dt * dt * dt / 24.0 * (A[v] + 3.0 * C2[v] + E1[v]);
      GT[v] += dt * dt * dt / 24.0 * (B[v] + 3.0 * D2[v] + G1b[v]);
    }
  }
}

/* ------------------------------------------------------------------ */
/* Sec. 3.3, Step 5(b): largest mu in [0,1] keeping the average        */
/* pressure of mu q^c + (1-mu) q^LxF above eps_p = min(eps0, p^LxF/2).  */
/* rho p/(g-1) - eps_p rho/(g-1) is quadratic in mu; its unique root in */
/* (0,1) is taken in the cancellation-free form 2h0/(-h1+sqrt(h1^2-4h0h2)). */
/* ------------------------------------------------------------------ */
double orc_mu_solve(double g, double eps0, const double* ql, const double* qc) {
  double pl = pressure(g, ql);
  if (!(ql[0] > 0.0) || !(pl > 0.0)) return 0.0;
  double eps_p = fmin(eps0, 0.5 * pl);
  double kappa = eps_p / (g - 1.0);
  double d[4];
  for (int v = 0; v < NV; ++v) d[v] = qc[v] - ql[v];
  /* h(mu) = rho E - |M|^2/2 - kappa rho along q(mu) = ql + mu d */
  double h0 = ql[0] * ql[3] - 0.5 * (ql[1] * ql[1] + ql[2] * ql[2]) - kappa * ql[0];
  double h1 = ql[0] * d[3] + d[0] * ql[3] - (ql[1] * d[1] + ql[2] * d[2]) - kappa * d[0];
  double h2 = d[0] * d[3] - 0.5 * (d[1] * d[1] + d[2] * d[2]);
  double h_one = h0 + h1 + h2;
  if (qc[0] > 0.0 && h_one >= 0.0) return 1.0;
  double disc = h1 * h1 - 4.0 * h0 * h2;
  if (disc < 0.0) disc = 0.0;
  double den = -h1 + sqrt(disc);
  if (!(den > 0.0)) return 0.0;
  double mu = 2.0 * h0 / den;
  if (mu > 1.0) mu = 1.0;
  if (mu < 0.0) mu = 0.0;
  return mu;
}

/* ------------------------------------------------------------------ */
/* Sec. 4.1: shock-capturing limiter on the primitive variables.       */
/* ------------------------------------------------------------------ */
static void primitive(double g, const double* q, double* w) {
  w[0] = q[0]; w[1] = q[1] / q[0]; w[2] = q[2] / q[0]; w[3] = pressure(g, q);
}

static double shock_theta_element(const orc_solver* s, const double* Q, int i) {
  const orc_mesh* m = s->m;
  int ML = s->ML, E = s->E;
  double g = s->gamma;
  const double* Qi = Q + (size_t)i * NV * ML;
  double qbar[4] = {Qi[0], Qi[ML], Qi[2 * ML], Qi[3 * ML]};
  if (!(qbar[0] > 0.0)) return 0.0;
  double wbar[4];
  primitive(g, qbar, wbar);
  double alpha = s->alpha0 * pow(m->sdx[i], 1.5);
  double Mx[4], Mn[4];
  for (int c = 0; c < 4; ++c) { Mx[c] = wbar[c] + alpha; Mn[c] = wbar[c] - alpha; }
  for (int k = 0; k < E; ++k) {
    int j = m->nbr[i * E + k];
    double qj[4];
    if (j >= 0) {
      const double* Qj = Q + (size_t)j * NV * ML;
      qj[0] = Qj[0]; qj[1] = Qj[ML]; qj[2] = Qj[2 * ML]; qj[3] = Qj[3 * ML];
    } else {
      const double* n = m->nrm + ((size_t)i * E + k) * 2;
      double ln = sqrt(n[0] * n[0] + n[1] * n[1]);
      double nh[2] = {n[0] / ln, n[1] / ln};
      boundary_state(m->bc[i * E + k], nh, qbar, qj, s->qinf, 0);
    }
    if (!(qj[0] > 0.0)) continue;
    double wj[4];
    primitive(g, qj, wj);
    for (int c = 0; c < 4; ++c) {
      if (wj[c] > Mx[c]) Mx[c] = wj[c];
      if (wj[c] < Mn[c]) Mn[c] = wj[c];
    }
  }
  double hmax[4], hmin[4];
  for (int c = 0; c < 4; ++c) { hmax[c] = -1e300; hmin[c] = 1e300; }
  for (int p = 0; p < s->NPT; ++p) {
    double q[4], w[4];
    eval_point(s, Qi, s->phi[p], q);
    if (!(q[0] > 0.0)) return 0.0;
    primitive(g, q, w);
    for (int c = 0; c < 4; ++c) {
      if (w[c] > hmax[c]) hmax[c] = w[c];
      if (w[c] < hmin[c]) hmin[c] = w[c];
    }
  }
  double th = 1.0;
  for (int c = 0; c < 4; ++c) {
    if (hmax[c] > wbar[c]) { double t = (Mx[c] - wbar[c]) / (hmax[c] - wbar[c]); if (t < th) th = t; }
    if (hmin[c] < wbar[c]) { double t = (wbar[c] - Mn[c]) / (wbar[c] - hmin[c]); if (t < th) th = t; }
  }
  if (th < 0.0) th = 0.0;
  return th;
}

void orc_shock_limit(const orc_solver* s, double* Q, double* theta) {
  int N = s->m->N, ML = s->ML;
  double* th = malloc(sizeof(double) * (size_t)N);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < N; ++i) th[i] = shock_theta_element(s, Q, i);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < N; ++i) {
    double* Qi = Q + (size_t)i * NV * ML;
    if (th[i] < 1.0)
      for (int v = 0; v < NV; ++v)
        for (int l = 1; l < ML; ++l) Qi[v * ML + l] *= th[i];
    if (theta) theta[i] = th[i];
  }
  free(th);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.3 Steps 4-5 on one element, given the outward (eps_ik applied)  */
/* f^LxW and f^LxF of its E edges: Gamma_i, the density Lambda_ik of the  */
/* four cases, the Lax-Friedrichs state, the 2^E - 1 box corners and mu_c,*/
/* and the proposals Lambda_ik * min_{c containing k} mu_c.  Returns 1 if */
/* Gamma^rho < 0 (the CFL bound of the low-order scheme is violated).     */
/* ------------------------------------------------------------------ */
int orc_flux_limit_cell(double g, double eps0, int E, double T, double dt, const double* qbar,
                        const double* fWp, const double* fFp, double* prop) {
  const double(*fW)[4] = (const double(*)[4])fWp;
  const double(*fF)[4] = (const double(*)[4])fFp;
  /* Gamma_i = |T_i|/dt qbar - sum_k f^LxF_k */
  double Gam[4];
  for (int v = 0; v < NV; ++v) {
    double a = T / dt * qbar[v];
    for (int k = 0; k < E; ++k) a -= fF[k][v];
    Gam[v] = a;
  }
  /* Step 4: sort the density flux differences Delta f_k = f^LxF - f^LxW;
   * the negative ones share Lambda = Gamma^rho / |their sum| (cases 1-4) */
  double df[MAXE];
  int ord[MAXE];
  for (int k = 0; k < E; ++k) { df[k] = fF[k][0] - fW[k][0]; ord[k] = k; }
  for (int a = 1; a < E; ++a)
    for (int b = a; b > 0 && df[ord[b]] < df[ord[b - 1]]; --b) { int t = ord[b]; ord[b] = ord[b - 1]; ord[b - 1] = t; }
  double negsum = 0.0;
  int nneg = 0;
  for (int a = 0; a < E; ++a) if (df[ord[a]] < 0.0) { negsum += df[ord[a]]; ++nneg; }
  double rho_lxf = dt / T * Gam[0];
  double eps_r = fmin(eps0, 0.5 * rho_lxf);
  if (eps_r < 0.0) eps_r = 0.0;
  double lneg = 1.0;
  if (nneg > 0) {
    lneg = (Gam[0] - T / dt * eps_r) / fabs(negsum);
    if (lneg > 1.0) lneg = 1.0;
    if (lneg < 0.0) lneg = 0.0;
  }
  double Lam[MAXE];
  for (int k = 0; k < E; ++k) Lam[k] = df[k] < 0.0 ? lneg : 1.0;
  /* Step 5: Lax-Friedrichs average state and the 2^E - 1 box corners */
  double qlxf[4];
  for (int v = 0; v < NV; ++v) {
    double a = 0.0;
    for (int k = 0; k < E; ++k) a += fF[k][v];
    qlxf[v] = qbar[v] - dt / T * a;
  }
  double mmin[MAXE];
  for (int k = 0; k < E; ++k) mmin[k] = 1.0;
  for (int c = 1; c < (1 << E); ++c) {
    double qc[4];
    for (int v = 0; v < NV; ++v) {
      double a = 0.0;
      for (int k = 0; k < E; ++k) {
        double al = (c >> k) & 1 ? Lam[k] : 0.0;
        a += al * fW[k][v] + (1.0 - al) * fF[k][v];
      }
      qc[v] = qbar[v] - dt / T * a;
    }
    double mu = orc_mu_solve(g, eps0, qlxf, qc);
    for (int k = 0; k < E; ++k)
      if ((c >> k) & 1 && mu < mmin[k]) mmin[k] = mu;
  }
  for (int k = 0; k < E; ++k) prop[k] = Lam[k] * mmin[k];
  return Gam[0] < 0.0;
}

/* ------------------------------------------------------------------ */
/* One time step: Sec. 3.3 "Putting it all together", Steps 1-6, then  */
/* the shock-capturing limiter (outline Step 5).                        */
/* ------------------------------------------------------------------ */
int orc_step(orc_solver* s, double* Q, double dt_in, double cfl, double* diag,
             double* theta_mom, double* theta_sc, double* theta_edge) {
  const orc_mesh* m = s->m;
  int N = m->N, E = s->E, ML = s->ML, MQ = s->MQ, NQ = s->NQ, ne = m->nedges;
  double g = s->gamma;
  int status = 0;

  /* Step 1 (element loop): moment limiter */
  int nmom = 0;
  {
    int st = 0;
#pragma omp parallel for reduction(| : st) reduction(+ : nmom) schedule(static)
    for (int i = 0; i < N; ++i) {
      int sti = 0;
      double t = moment_limit_element(s, Q + (size_t)i * NV * ML, &sti);
      if (theta_mom) theta_mom[i] = t;
      if (t < 1.0) ++nmom;
      st |= sti;
    }
    status |= st;
  }
  /* global wave speed and time step */
  double sw = orc_wave_speed(s, Q);
  double dt = dt_in > 0.0 ? dt_in : cfl * m->hmin / sw;
  s->last_dt = dt;

  /* Step 2 (element loop): time-averaged fluxes, volume integrals, traces */
#pragma omp parallel for schedule(static)
  for (int i = 0; i < N; ++i) {
    double q[MAXPTS][4], qt[MAXPTS][4], qtt[MAXPTS][4], FT[MAXPTS][4], GT[MAXPTS][4], qttt[MAXPTS][4];
    double V[MAXML][4];
    ck_element(s, Q + (size_t)i * NV * ML, i, dt, q, qt, qtt, FT, GT, V, qttt);
    for (int l = 0; l < ML; ++l)
      for (int v = 0; v < NV; ++v) s->V[((size_t)i * ML + l) * NV + v] = V[l][v];
    for (int k = 0; k < E; ++k)
      for (int p = 0; p < MQ; ++p) {
        size_t t = (((size_t)i * E + k) * MQ + p) * NV;
        int src = NQ + k * MQ + p;
        for (int v = 0; v < NV; ++v) {
          s->tq[t + v] = q[src][v]; s->tqt[t + v] = qt[src][v]; s->tqtt[t + v] = qtt[src][v];
          s->tqttt[t + v] = qttt[src][v];
          s->tF[t + v] = FT[src][v]; s->tG[t + v] = GT[src][v];
        }
      }
  }

  /* Step 3 (edge loop): high-order flux at the edge points, f^LxW, f^LxF */
#pragma omp parallel for schedule(static)
  for (int e = 0; e < ne; ++e) {
    int i = m->e_i[e], ki = m->e_ki[e], j = m->e_j[e], kj = m->e_kj[e];
    const double* n = m->nrm + ((size_t)i * E + ki) * 2;   /* n_e, outward for i_e */
    double ln = sqrt(n[0] * n[0] + n[1] * n[1]);
    double nh[2] = {n[0] / ln, n[1] / ln};
    int bc = m->bc[i * E + ki];
    double fw[4] = {0, 0, 0, 0};
    for (int p = 0; p < MQ; ++p) {
      size_t ti = (((size_t)i * E + ki) * MQ + p) * NV;
      const double *qm = s->tq + ti, *Fm = s->tF + ti, *Gm = s->tG + ti;
      double qp[4], Fp[4], Gp[4];
      if (j >= 0) {
        /* the neighbour runs along the shared edge in the opposite direction */
        size_t tj = (((size_t)j * E + kj) * MQ + (MQ - 1 - p)) * NV;
        for (int v = 0; v < NV; ++v) { qp[v] = s->tq[tj + v]; Fp[v] = s->tF[tj + v]; Gp[v] = s->tG[tj + v]; }
      } else {
        double qtp[4], qttp[4], qtttp[4];
        boundary_state(bc, nh, qm, qp, s->qinf, 0);
        boundary_state(bc, nh, s->tqt + ti, qtp, s->qinf, 1);
        boundary_state(bc, nh, s->tqtt + ti, qttp, s->qinf, 1);
        boundary_state(bc, nh, s->tqttt + ti, qtttp, s->qinf, 1);
        ft_from_derivs(g, dt, qp, qtp, qttp, s->ck_order == 4 ? qtttp : NULL, Fp, Gp);
      }
      double* fs = s->fstar + ((size_t)e * MQ + p) * NV;
      /* dissipation speed: local Lax-Friedrichs speed of the two traces,
       * bounded by the global s (or the global s itself, literal reading) */
      double sp = sw;
      if (!s->llf_global) {
        double am = wave_speed_point(g, qm), ap = wave_speed_point(g, qp);
        double a = am > ap ? am : ap;
        if (a < sp) sp = a;
      }
      for (int v = 0; v < NV; ++v) {
        /* Eq. LLF times the edge length */
        fs[v] = 0.5 * (n[0] * (Fp[v] + Fm[v]) + n[1] * (Gp[v] + Gm[v])) - 0.5 * sp * ln * (qp[v] - qm[v]);
        fw[v] += 0.5 * s->gw[p] * fs[v];
      }
    }
    /* Lax-Friedrichs flux from the cell averages (Sec. 3.2) */
    const double* Qi = Q + (size_t)i * NV * ML;
    double qi[4] = {Qi[0], Qi[ML], Qi[2 * ML], Qi[3 * ML]}, qj[4];
    if (j >= 0) {
      const double* Qj = Q + (size_t)j * NV * ML;
      qj[0] = Qj[0]; qj[1] = Qj[ML]; qj[2] = Qj[2 * ML]; qj[3] = Qj[3 * ML];
    } else {
      boundary_state(bc, nh, qi, qj, s->qinf, 0);
    }
    double Fi[4], Gi[4], Fj[4], Gj[4];
    orc_flux(g, qi, Fi, Gi);
    orc_flux(g, qj, Fj, Gj);
    for (int v = 0; v < NV; ++v) {
      s->flxw[(size_t)e * NV + v] = fw[v];
      s->flxf[(size_t)e * NV + v] =
          0.5 * (n[0] * (Fj[v] + Fi[v]) + n[1] * (Gj[v] + Gi[v])) - 0.5 * ln * sw * (qj[v] - qi[v]);
    }
  }

  /* Steps 4-5 (element loop): Lambda proposals per element edge */
  int cfl_bad = 0;
#pragma omp parallel for reduction(| : cfl_bad) schedule(static)
  for (int i = 0; i < N; ++i) {
    const double* Qi = Q + (size_t)i * NV * ML;
    double qbar[4] = {Qi[0], Qi[ML], Qi[2 * ML], Qi[3 * ML]};
    double fW[MAXE][4], fF[MAXE][4];
    for (int k = 0; k < E; ++k) {
      int e = m->edge_of[i * E + k];
      double ek = m->eps[i * E + k];
      for (int v = 0; v < NV; ++v) {
        fW[k][v] = ek * s->flxw[(size_t)e * NV + v];
        fF[k][v] = ek * s->flxf[(size_t)e * NV + v];
      }
    }
    if (orc_flux_limit_cell(g, s->eps0, E, m->area[i], dt, qbar, &fW[0][0], &fF[0][0],
                            s->prop + (size_t)i * E))
      cfl_bad = 1;
  }
  if (cfl_bad) status |= ORC_ST_CFL;

  /* Step 6 (element loop): theta_k = Lambda_e (min over both sides) and update */
  int nedge_lim = 0;
  double* Qn = malloc(sizeof(double) * (size_t)N * NV * ML);
#pragma omp parallel for reduction(+ : nedge_lim) schedule(static)
  for (int i = 0; i < N; ++i) {
    const double* Qi = Q + (size_t)i * NV * ML;
    double* Qo = Qn + (size_t)i * NV * ML;
    double T = m->area[i];
    double Eint[MAXML][4];
    for (int l = 0; l < ML; ++l) for (int v = 0; v < NV; ++v) Eint[l][v] = 0.0;
    double avg_upd[4] = {0, 0, 0, 0};
    for (int k = 0; k < E; ++k) {
      int e = m->edge_of[i * E + k];
      double ek = m->eps[i * E + k];
      int j = m->nbr[i * E + k];
      double th = s->prop[(size_t)i * E + k];
      if (j >= 0) { double o = s->prop[(size_t)j * E + m->nbk[i * E + k]]; if (o < th) th = o; }
      if (theta_edge) theta_edge[(size_t)i * E + k] = th;
      if (th < 1.0 && ek > 0) ++nedge_lim;
      for (int v = 0; v < NV; ++v)
        avg_upd[v] += ek * (th * s->flxw[(size_t)e * NV + v] + (1.0 - th) * s->flxf[(size_t)e * NV + v]);
      /* edge integral of phi_l F*.n over this edge; points seen from element i */
      for (int p = 0; p < MQ; ++p) {
        int pe = ek > 0 ? p : MQ - 1 - p;   /* index along the owner's direction */
        const double* fs = s->fstar + ((size_t)e * MQ + pe) * NV;
        int pt = NQ + k * MQ + p;
        for (int l = 0; l < ML; ++l)
          for (int v = 0; v < NV; ++v) Eint[l][v] += 0.5 * s->gw[p] * s->phi[pt][l] * ek * fs[v];
      }
    }
    for (int v = 0; v < NV; ++v) {
      Qo[v * ML] = Qi[v * ML] - dt / T * avg_upd[v];
      for (int l = 1; l < ML; ++l)
        Qo[v * ML + l] = Qi[v * ML + l] + dt / T * (s->V[((size_t)i * ML + l) * NV + v] - Eint[l][v]);
    }
  }
  memcpy(Q, Qn, sizeof(double) * (size_t)N * NV * ML);
  free(Qn);

  /* outline Step 5: shock-capturing limiter on the new state */
  int nsc = 0;
  if (s->shock_limiter) {
    double* th = theta_sc ? theta_sc : malloc(sizeof(double) * (size_t)N);
    orc_shock_limit(s, Q, th);
    for (int i = 0; i < N; ++i) if (th[i] < 1.0) ++nsc;
    if (!theta_sc) free(th);
  } else if (theta_sc) {
    for (int i = 0; i < N; ++i) theta_sc[i] = 1.0;
  }

  if (diag) {
    double mr = 1e300, mp = 1e300, tot[4] = {0, 0, 0, 0};
    for (int i = 0; i < N; ++i) {
      const double* Qi = Q + (size_t)i * NV * ML;
      double qb[4] = {Qi[0], Qi[ML], Qi[2 * ML], Qi[3 * ML]};
      double pb = pressure(g, qb);
      if (qb[0] < mr) mr = qb[0];
      if (pb < mp) mp = pb;
      for (int v = 0; v < NV; ++v) tot[v] += m->area[i] * qb[v];
      for (int v = 0; v < NV; ++v) if (!isfinite(Qi[v * ML])) status |= ORC_ST_NAN;
    }
    for (int c = 0; c < ORC_DIAG_LEN; ++c) diag[c] = 0.0;
    diag[ORC_D_S] = sw; diag[ORC_D_DT] = dt; diag[ORC_D_MINRHO] = mr; diag[ORC_D_MINP] = mp;
    diag[ORC_D_MASS] = tot[0]; diag[ORC_D_MOMX] = tot[1]; diag[ORC_D_MOMY] = tot[2];
    diag[ORC_D_ENERGY] = tot[3]; diag[ORC_D_NMOM] = nmom; diag[ORC_D_NEDGE] = nedge_lim;
    diag[ORC_D_NSC] = nsc; diag[ORC_D_STATUS] = status;
  }
  return status;
}

/* ------------------------------------------------------------------ */
/* Learned troubled-cell indicator, FP64 reference of the network and  */
/* its features (the GPU trains and evaluates them in FP32 / BF16).    */
/* MLP 24 -> 64 ReLU -> 64 ReLU -> 1 sigmoid; parameters W1[24][64],   */
/* b1[64], W2[64][64], b2[64], w3[64], b3.                              */
/* ------------------------------------------------------------------ */
#define MI 24
#define MH 64
double orc_mlp_loss_grad(const double* P, const double* X, const double* y, int B, double* grad, double* yhat) {
  const double *W1 = P, *b1 = P + MI * MH, *W2 = b1 + MH, *b2 = W2 + MH * MH, *w3 = b2 + MH, *b3 = w3 + MH;
  double *gW1 = 0, *gb1 = 0, *gW2 = 0, *gb2 = 0, *gw3 = 0, *gb3 = 0;
  if (grad) {
    memset(grad, 0, sizeof(double) * (MI * MH + MH + MH * MH + MH + MH + 1));
    gW1 = grad; gb1 = gW1 + MI * MH; gW2 = gb1 + MH; gb2 = gW2 + MH * MH; gw3 = gb2 + MH; gb3 = gw3 + MH;
  }
  double loss = 0.0;
  for (int r = 0; r < B; ++r) {
    const double* x = X + (size_t)r * MI;
    double z1[MH], h1[MH], z2[MH], h2[MH];
    for (int j = 0; j < MH; ++j) {
      double a = b1[j];
      for (int i = 0; i < MI; ++i) a += x[i] * W1[i * MH + j];
      z1[j] = a; h1[j] = a > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < MH; ++j) {
      double a = b2[j];
      for (int k = 0; k < MH; ++k) a += h1[k] * W2[k * MH + j];
      z2[j] = a; h2[j] = a > 0.0 ? a : 0.0;
    }
    double z3 = b3[0];
    for (int j = 0; j < MH; ++j) z3 += h2[j] * w3[j];
    double s = 1.0 / (1.0 + exp(-z3));
    if (yhat) yhat[r] = s;
    if (!y) continue;
    double d = s - y[r];
    loss += d * d / B;
    if (!grad) continue;
    double dz3 = 2.0 * d * s * (1.0 - s) / B;
    gb3[0] += dz3;
    double dz2[MH], dz1[MH];
    for (int j = 0; j < MH; ++j) {
      gw3[j] += h2[j] * dz3;
      dz2[j] = z2[j] > 0.0 ? dz3 * w3[j] : 0.0;
      gb2[j] += dz2[j];
    }
    for (int k = 0; k < MH; ++k) {
      double a = 0.0;
      for (int j = 0; j < MH; ++j) {
        gW2[k * MH + j] += h1[k] * dz2[j];
        a += W2[k * MH + j] * dz2[j];
      }
      dz1[k] = z1[k] > 0.0 ? a : 0.0;
      gb1[k] += dz1[k];
    }
    for (int i = 0; i < MI; ++i)
      for (int j = 0; j < MH; ++j) gW1[i * MH + j] += x[i] * dz1[j];
  }
  return loss;
}

static double clip8(double v) { return v > 8.0 ? 8.0 : (v < -8.0 ? -8.0 : v); }

/* Features of every cell of Q (the state at the shock limiter's input). */
void orc_features(const orc_solver* s, const double* Q, double* F) {
  const orc_mesh* m = s->m;
  int ML = s->ML, E = s->E;
  double g = s->gamma;
  for (int i = 0; i < m->N; ++i) {
    const double* Qi = Q + (size_t)i * NV * ML;
    double* f = F + (size_t)i * MI;
    double r = Qi[0], e = Qi[3 * ML];
    double u = Qi[ML] / r, v = Qi[2 * ML] / r;
    double p = (g - 1.0) * (e - 0.5 * r * (u * u + v * v));
    if (p < 0.0) p = 0.0;
    double U = sqrt(u * u + v * v) + sqrt(g * p / r);
    double mi = 1.0 / (r * U > 1e-30 ? r * U : 1e-30);
    for (int l = 1; l <= 5; ++l) {
      f[l - 1] = l < ML ? Qi[l] / r : 0.0;
      f[4 + l] = l < ML ? Qi[3 * ML + l] / e : 0.0;
    }
    f[10] = Qi[ML + 1] * mi; f[11] = Qi[2 * ML + 1] * mi; f[12] = Qi[ML + 2] * mi; f[13] = Qi[2 * ML + 2] * mi;
    for (int k = 0; k < 4; ++k) { f[14 + k] = 0.0; f[18 + k] = 0.0; }
    double qbar[4] = {Qi[0], Qi[ML], Qi[2 * ML], Qi[3 * ML]};
    for (int k = 0; k < E; ++k) {
      int j = m->nbr[i * E + k];
      double qn[4];
      if (j >= 0) {
        const double* Qj = Q + (size_t)j * NV * ML;
        qn[0] = Qj[0]; qn[1] = Qj[ML]; qn[2] = Qj[2 * ML]; qn[3] = Qj[3 * ML];
      } else {
        const double* n = m->nrm + ((size_t)i * E + k) * 2;
        double ln = sqrt(n[0] * n[0] + n[1] * n[1]);
        double nh[2] = {n[0] / ln, n[1] / ln};
        boundary_state(m->bc[i * E + k], nh, qbar, qn, s->qinf, 0);
      }
      if (qn[0] > 0.0) { f[14 + k] = qn[0] / r - 1.0; f[18 + k] = qn[3] / e - 1.0; }
    }
    double al = s->alpha0 * pow(m->sdx[i], 1.5);
    f[22] = al / r;
    f[23] = p / ((g - 1.0) * e);
    for (int k = 0; k < MI; ++k) f[k] = clip8(f[k]);
  }
}
