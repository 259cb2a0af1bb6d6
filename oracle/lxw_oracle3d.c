/*
 * lxw_oracle3d.c -- plain FP64 oracle of the LxW-DG step on 3D Cartesian
 * meshes.  TEST INFRASTRUCTURE ONLY (see lxw_oracle3d.h for what it follows
 * and the conventions it shares with the GPU library by documentation).
 *
 * Readings beyond the 2D oracle's (its header lists those, they carry over):
 *  - dt = cfl * hmin / s with hmin = min_i 3 |K_i| / |dK_i| (half the side
 *    of a cube, as min 2|T|/P is half the side of a square in 2D).
 *  - shock limiter alpha = alpha0 * dx^1.5 with dx = |K|^(1/3) (the side of
 *    a cube; the 2D oracle takes the side of a square).
 *  - the flux derivatives F'(q) w and F''(q)(w, w) + F'(q) b come from the
 *    Taylor coefficients of F along q + t w + t^2 b / 2 (series arithmetic
 *    of the flux formula), not from hand-derived Jacobians.
 *  - the moment limiter's pressure step is the secant of Lemma 1 only.
 *  - q_t = -div F^h and q_tt = -div F_t^h lie in the modal space (degree
 *    deg - 1): they are evaluated at the interior points, projected onto the
 *    modes with the interior rule and evaluated from the modes elsewhere.
 *  - tetrahedra: the interior and face rules are conical products of
 *    Gauss-Jacobi rules with deg + 1 points per direction, exact to degree
 *    2 deg + 1 like the hexahedra's tensor rules (the mass matrix is
 *    exact); a
 *    face's points are generated from its vertices in the order of their
 *    (periodically identified) ids, so both cells meet them in one order.
 */
#include "lxw_oracle3d.h"
#include "lxw_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NV3 5
#define MAXML3 20                 /* modes of degree 3 */
#define MAXN3 4                   /* points per direction (degree 3) */
#define MAXQ3 64                  /* interior points: (deg+1)^3 */
#define MAXF3 (MAXN3 * MAXN3)     /* points per face */
#define MAXPTS3 (MAXQ3 + 6 * MAXF3)
#define MAXNJ3 6                  /* projection points per direction */
#define MAXPJ3 (MAXNJ3 * MAXNJ3 * MAXNJ3)

enum { B3_PERIODIC = 0, B3_REFLECT = 1, B3_TRANSPARENT = 2 };
enum { ST3_NONPOSITIVE = 1, ST3_CFL = 2, ST3_NAN = 4 };

/* ------------------------------------------------------------------ */
/* Basis: products of normalised Legendre polynomials                  */
/* ------------------------------------------------------------------ */
static void leg3(int n, double x, double* v, double* d) {
  /* L_k = sqrt(2k+1) P_k and derivatives, k = 0..n */
  double p[8], dp[8];
  p[0] = 1.0; dp[0] = 0.0;
  if (n >= 1) { p[1] = x; dp[1] = 1.0; }
  for (int k = 2; k <= n; ++k) {
    p[k] = ((2.0 * k - 1.0) * x * p[k - 1] - (k - 1.0) * p[k - 2]) / k;
    dp[k] = dp[k - 2] + (2.0 * k - 1.0) * p[k - 1];
  }
  for (int k = 0; k <= n; ++k) { v[k] = sqrt(2.0 * k + 1.0) * p[k]; d[k] = sqrt(2.0 * k + 1.0) * dp[k]; }
}

int orc3_num_modes(int deg) { return (deg + 1) * (deg + 2) * (deg + 3) / 6; }

void orc3_mode_exponents(int deg, int* abc) {
  int l = 0;
  for (int t = 0; t <= deg; ++t)
    for (int a = t; a >= 0; --a)
      for (int b = t - a; b >= 0; --b) {
        abc[3 * l] = a; abc[3 * l + 1] = b; abc[3 * l + 2] = t - a - b;
        ++l;
      }
}

int orc3_basis_eval(int deg, int npts, const double* xi, const double* eta, const double* zeta, double* phi,
                    double* dxi, double* deta, double* dzeta) {
  int ML = orc3_num_modes(deg);
  int abc[3 * MAXML3];
  orc3_mode_exponents(deg, abc);
  for (int p = 0; p < npts; ++p) {
    double vx[8], dx[8], vy[8], dy[8], vz[8], dz[8];
    leg3(deg, xi[p], vx, dx);
    leg3(deg, eta[p], vy, dy);
    leg3(deg, zeta[p], vz, dz);
    for (int l = 0; l < ML; ++l) {
      int a = abc[3 * l], b = abc[3 * l + 1], c = abc[3 * l + 2];
      if (phi) phi[p * ML + l] = vx[a] * vy[b] * vz[c];
      if (dxi) dxi[p * ML + l] = dx[a] * vy[b] * vz[c];
      if (deta) deta[p * ML + l] = vx[a] * dy[b] * vz[c];
      if (dzeta) dzeta[p * ML + l] = vx[a] * vy[b] * dz[c];
    }
  }
  return ML;
}

/* ------------------------------------------------------------------ */
/* Euler flux (Sec. 1.1 in three dimensions) and its Taylor series     */
/* ------------------------------------------------------------------ */
static double pressure3(double g, const double* q) {
  return (g - 1.0) * (q[4] - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0]);
}

void orc3_flux(double g, const double* q, double* F) {
  double p = pressure3(g, q);
  double u[3] = {q[1] / q[0], q[2] / q[0], q[3] / q[0]};
  for (int d = 0; d < 3; ++d) {
    double* Fd = F + 5 * d;
    Fd[0] = q[1 + d];
    for (int e = 0; e < 3; ++e) Fd[1 + e] = q[1 + e] * u[d] + (e == d ? p : 0.0);
    Fd[4] = (q[4] + p) * u[d];
  }
}

/* truncated power series of order K: c[0..K] */
static void s_mul(int K, const double* a, const double* b, double* r) {
  for (int k = 0; k <= K; ++k) {
    double s = 0.0;
    for (int i = 0; i <= k; ++i) s += a[i] * b[k - i];
    r[k] = s;
  }
}
static void s_inv(int K, const double* a, double* r) {
  r[0] = 1.0 / a[0];
  for (int k = 1; k <= K; ++k) {
    double s = 0.0;
    for (int i = 1; i <= k; ++i) s += a[i] * r[k - i];
    r[k] = -s / a[0];
  }
}

void orc3_flux_series(double g, int K, const double* qs, double* Fs) {
  /* series of each conserved variable */
  double q[5][4], u[3][4], ri[4], ke[4], p[4], t[4];
  for (int v = 0; v < 5; ++v)
    for (int k = 0; k <= K; ++k) q[v][k] = qs[k * 5 + v];
  s_inv(K, q[0], ri);
  for (int d = 0; d < 3; ++d) s_mul(K, q[1 + d], ri, u[d]);
  for (int k = 0; k <= K; ++k) ke[k] = 0.0;
  for (int d = 0; d < 3; ++d) {
    s_mul(K, q[1 + d], u[d], t);
    for (int k = 0; k <= K; ++k) ke[k] += 0.5 * t[k];
  }
  for (int k = 0; k <= K; ++k) p[k] = (g - 1.0) * (q[4][k] - ke[k]);
  for (int d = 0; d < 3; ++d) {
    double mu[4], ep[4];
    for (int k = 0; k <= K; ++k) Fs[(k * 3 + d) * 5 + 0] = q[1 + d][k];
    for (int e = 0; e < 3; ++e) {
      s_mul(K, q[1 + e], u[d], mu);
      for (int k = 0; k <= K; ++k) Fs[(k * 3 + d) * 5 + 1 + e] = mu[k] + (e == d ? p[k] : 0.0);
    }
    for (int k = 0; k <= K; ++k) t[k] = q[4][k] + p[k];
    s_mul(K, t, u[d], ep);
    for (int k = 0; k <= K; ++k) Fs[(k * 3 + d) * 5 + 4] = ep[k];
  }
}

static double wave_speed3(double g, const double* q) {
  if (!(q[0] > 0.0)) return 0.0;
  double p = pressure3(g, q);
  double u = q[1] / q[0], v = q[2] / q[0], w = q[3] / q[0];
  double c = p > 0.0 ? sqrt(g * p / q[0]) : 0.0;
  return sqrt(u * u + v * v + w * w) + c;
}

/* ------------------------------------------------------------------ */
/* Tetrahedra: reference T0 = {r, s, t >= 0, r + s + t <= 1}.  Rules    */
/* by the collapsed map r = u, s = v (1 - u), t = w (1 - u) (1 - v)     */
/* (Stroud's conical product): the map's Jacobian (1 - u)^2 (1 - v) is  */
/* taken into the weight functions of Gauss rules in u and v, so n      */
/* points per direction integrate total degree 2n - 1 exactly.          */
/* Triangle faces: r = u, s = v (1 - u), weight (1 - u) in u.  Weights  */
/* sum to 1 (the rule of (1/|T0|) Int).  The basis is the Gram-Schmidt  */
/* orthonormalisation (under (1/|T0|) Int) of the monomials r^a s^b t^c  */
/* in the mode order of the hexahedra.                                  */
/* ------------------------------------------------------------------ */

/* Jacobi polynomial P_n^(alpha, 0)(x) and its derivative by the three-term
 * recurrence in n (its derivative by differentiating the recurrence). */
static void jacobi_p(int n, double al, double x, double* p, double* dp) {
  double p0 = 1.0, d0 = 0.0;
  if (n == 0) { *p = p0; *dp = d0; return; }
  double p1 = 0.5 * ((al + 2.0) * x + al), d1 = 0.5 * (al + 2.0);
  for (int k = 2; k <= n; ++k) {
    double sk = 2.0 * k + al;
    double A = (sk - 1.0) * sk * (sk - 2.0), B = (sk - 1.0) * al * al;
    double C = 2.0 * (k + al - 1.0) * (k - 1.0) * sk, D = 2.0 * k * (k + al) * (sk - 2.0);
    double p2 = ((A * x + B) * p1 - C * p0) / D;
    double d2 = ((A * x + B) * d1 + A * p1 - C * d0) / D;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *p = p1; *dp = d1;
}

/* n-point Gauss rule on [0, 1] for the weight (1 - u)^al: the nodes are the
 * roots of P_n^(al, 0) mapped from [-1, 1], found one after another by
 * Newton's method with the roots already found divided out (Maehly) and
 * sorted ascending; each
 * weight integrates its node's Lagrange polynomial against the weight
 * function exactly (Gauss-Legendre with n + 2 points).  Unnormalised. */
static void gauss_jacobi01(int n, double al, double* u, double* w) {
  double x[8];
  for (int j = 0; j < n; ++j) {
    double z = -cos(3.14159265358979323846 * (j + 0.75) / (n + 0.5));
    if (j > 0 && z <= x[j - 1]) z = x[j - 1] + 1e-3;
    for (int it = 0; it < 200; ++it) {
      double p, dp, sdef = 0.0;
      jacobi_p(n, al, z, &p, &dp);
      for (int i = 0; i < j; ++i) sdef += 1.0 / (z - x[i]);
      double dz = p / (dp - p * sdef);
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    x[j] = z;
  }
  for (int j = 1; j < n; ++j)   /* ascending (deflation may find the roots out of order) */
    for (int i = j; i > 0 && x[i] < x[i - 1]; --i) { double t = x[i]; x[i] = x[i - 1]; x[i - 1] = t; }
  double g[10], gw[10];
  orc_gauss_legendre(n + 2, g, gw);
  for (int j = 0; j < n; ++j) {
    double acc = 0.0;
    for (int q = 0; q < n + 2; ++q) {
      double l = pow(1.0 - g[q], al);
      for (int i = 0; i < n; ++i)
        if (i != j) l *= (g[q] - x[i]) / (x[j] - x[i]);
      acc += gw[q] * l;
    }
    u[j] = 0.5 * (x[j] + 1.0);
    w[j] = acc;
  }
}

static int tet_rule(int n, double* r, double* s, double* t, double* w) {
  double ua[8], uw[8], va[8], vw[8], wa[8], ww[8];
  gauss_jacobi01(n, 2.0, ua, uw);
  gauss_jacobi01(n, 1.0, va, vw);
  gauss_jacobi01(n, 0.0, wa, ww);
  int k = 0;
  double tot = 0.0;
  for (int c = 0; c < n; ++c)
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        double u = ua[a], v = va[b], x = wa[c];
        r[k] = u; s[k] = v * (1.0 - u); t[k] = x * (1.0 - u) * (1.0 - v);
        w[k] = uw[a] * vw[b] * ww[c];
        tot += w[k];
        ++k;
      }
  for (int i = 0; i < k; ++i) w[i] /= tot;
  return k;
}

static int tri_rule(int n, double* a, double* b, double* w) {
  double ua[8], uw[8], va[8], vw[8];
  gauss_jacobi01(n, 1.0, ua, uw);
  gauss_jacobi01(n, 0.0, va, vw);
  int k = 0;
  double tot = 0.0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      a[k] = ua[i]; b[k] = va[j] * (1.0 - ua[i]);
      w[k] = uw[i] * vw[j];
      tot += w[k];
      ++k;
    }
  for (int i = 0; i < k; ++i) w[i] /= tot;
  return k;
}

/* Gram-Schmidt coefficients: phi_l = sum_j C[l][j] r^a_j s^b_j t^c_j */
static void tet_basis_coeffs(int deg, double C[MAXML3][MAXML3]) {
  int ML = orc3_num_modes(deg), abc[3 * MAXML3];
  orc3_mode_exponents(deg, abc);
  double r[512], s[512], t[512], w[512];
  int nq = tet_rule(deg + 1, r, s, t, w);   /* exact to degree 2 deg + 1 >= 2 deg */
  static double M[512][MAXML3];
  for (int q = 0; q < nq; ++q)
    for (int j = 0; j < ML; ++j) M[q][j] = pow(r[q], abc[3 * j]) * pow(s[q], abc[3 * j + 1]) * pow(t[q], abc[3 * j + 2]);
  long double Cl[MAXML3][MAXML3];
  for (int l = 0; l < ML; ++l) {
    for (int j = 0; j < ML; ++j) Cl[l][j] = (j == l) ? 1.0L : 0.0L;
    for (int pass = 0; pass < 2; ++pass)   /* twice, for orthogonality to rounding */
      for (int m = 0; m < l; ++m) {
        long double ip = 0.0L;
        for (int q = 0; q < nq; ++q) {
          long double a = 0.0L, b = 0.0L;
          for (int j = 0; j < ML; ++j) { a += Cl[l][j] * M[q][j]; b += Cl[m][j] * M[q][j]; }
          ip += (long double)w[q] * a * b;
        }
        for (int j = 0; j < ML; ++j) Cl[l][j] -= ip * Cl[m][j];
      }
    long double nn = 0.0L;
    for (int q = 0; q < nq; ++q) {
      long double a = 0.0L;
      for (int j = 0; j < ML; ++j) a += Cl[l][j] * M[q][j];
      nn += (long double)w[q] * a * a;
    }
    for (int j = 0; j < ML; ++j) Cl[l][j] /= sqrtl(nn);
  }
  for (int l = 0; l < ML; ++l)
    for (int j = 0; j < ML; ++j) C[l][j] = (double)Cl[l][j];
}

/* the basis of coefficients C at npts points */
static void tet_basis_apply(int deg, double C[MAXML3][MAXML3], int npts, const double* r, const double* s,
                            const double* t, double* phi, double* dr, double* ds, double* dt) {
  int ML = orc3_num_modes(deg), abc[3 * MAXML3];
  orc3_mode_exponents(deg, abc);
  for (int p = 0; p < npts; ++p) {
    double m[MAXML3], mr[MAXML3], ms[MAXML3], mt[MAXML3];
    for (int j = 0; j < ML; ++j) {
      int a = abc[3 * j], b = abc[3 * j + 1], c = abc[3 * j + 2];
      double pr = pow(r[p], a), ps = pow(s[p], b), pt = pow(t[p], c);
      m[j] = pr * ps * pt;
      mr[j] = a ? a * pow(r[p], a - 1) * ps * pt : 0.0;
      ms[j] = b ? b * pr * pow(s[p], b - 1) * pt : 0.0;
      mt[j] = c ? c * pr * ps * pow(t[p], c - 1) : 0.0;
    }
    for (int l = 0; l < ML; ++l) {
      double v = 0, x = 0, y = 0, z = 0;
      for (int j = 0; j < ML; ++j) { v += C[l][j] * m[j]; x += C[l][j] * mr[j]; y += C[l][j] * ms[j]; z += C[l][j] * mt[j]; }
      if (phi) phi[p * ML + l] = v;
      if (dr) dr[p * ML + l] = x;
      if (ds) ds[p * ML + l] = y;
      if (dt) dt[p * ML + l] = z;
    }
  }
}

int orc3_tet_basis_eval(int deg, int npts, const double* r, const double* s, const double* t, double* phi,
                        double* dr, double* ds, double* dt) {
  double C[MAXML3][MAXML3];
  tet_basis_coeffs(deg, C);
  tet_basis_apply(deg, C, npts, r, s, t, phi, dr, ds, dt);
  return orc3_num_modes(deg);
}

/* ------------------------------------------------------------------ */
/* Meshes: per-element geometry for both kinds                          */
/* ------------------------------------------------------------------ */
enum { KIND3_HEX = 0, KIND3_TET = 1 };

struct orc3_mesh {
  int kind, E, N;
  int nx, ny, nz;       /* hexahedra */
  double *vol, *org, *Jm, *Ji;   /* [N], [N][3], [N][9] dx_a/dr_b, [N][9] dr_a/dx_b */
  double* nrm;          /* [N][E][3] outward normal scaled by the face area */
  int *nbr, *nbk;       /* [N][E]: neighbour (or -1 - bc) and its local face */
  int* canon;           /* tetrahedra [N][4][3]: the face's local vertices in id order */
  int nfaces;
  int *f_i, *f_k, *f_j; /* face: owner i, its local face k, neighbour j (or -1 - bc) */
  int* face_of;         /* [N][E] */
  double* eps;          /* [N][E] +1 owner side, -1 neighbour side */
  double hmin;
};

static orc3_mesh* mesh3_alloc(int kind, int N) {
  orc3_mesh* m = calloc(1, sizeof(orc3_mesh));
  m->kind = kind; m->E = kind == KIND3_HEX ? 6 : 4; m->N = N;
  int E = m->E;
  m->vol = malloc(sizeof(double) * N); m->org = malloc(sizeof(double) * 3 * N);
  m->Jm = malloc(sizeof(double) * 9 * N); m->Ji = malloc(sizeof(double) * 9 * N);
  m->nrm = malloc(sizeof(double) * 3 * E * N);
  m->nbr = malloc(sizeof(int) * E * N); m->nbk = malloc(sizeof(int) * E * N);
  m->f_i = malloc(sizeof(int) * E * N); m->f_k = malloc(sizeof(int) * E * N); m->f_j = malloc(sizeof(int) * E * N);
  m->face_of = malloc(sizeof(int) * E * N); m->eps = malloc(sizeof(double) * E * N);
  return m;
}

/* faces: owned by the cell of lower index (or the lower local face when a
 * cell meets itself across a period); boundary faces by their cell */
static void mesh3_faces(orc3_mesh* m) {
  int E = m->E, nf = 0;
  for (int i = 0; i < m->N; ++i)
    for (int k = 0; k < E; ++k) {
      int j = m->nbr[E * i + k], kj = m->nbk[E * i + k];
      if (j < 0 || i < j || (i == j && k < kj)) {
        m->f_i[nf] = i; m->f_k[nf] = k; m->f_j[nf] = j;
        m->face_of[E * i + k] = nf; m->eps[E * i + k] = 1.0;
        ++nf;
      }
    }
  for (int i = 0; i < m->N; ++i)
    for (int k = 0; k < E; ++k) {
      int j = m->nbr[E * i + k], kj = m->nbk[E * i + k];
      if (!(j < 0 || i < j || (i == j && k < kj))) {
        m->face_of[E * i + k] = m->face_of[E * j + kj];
        m->eps[E * i + k] = -1.0;
      }
    }
  m->nfaces = nf;
  m->hmin = 1e300;
  for (int i = 0; i < m->N; ++i) {
    double surf = 0.0;
    for (int k = 0; k < E; ++k) {
      const double* n = m->nrm + 3 * (E * i + k);
      surf += sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    }
    double hm = 3.0 * m->vol[i] / surf;
    if (hm < m->hmin) m->hmin = hm;
  }
}

orc3_mesh* orc3_mesh_cartesian(int nx, int ny, int nz, const double* box, const int* bc) {
  if (nx < 1 || ny < 1 || nz < 1) return NULL;
  int N = nx * ny * nz, n3[3] = {nx, ny, nz};
  orc3_mesh* m = mesh3_alloc(KIND3_HEX, N);
  m->nx = nx; m->ny = ny; m->nz = nz;
  double h[3] = {(box[1] - box[0]) / nx, (box[3] - box[2]) / ny, (box[5] - box[4]) / nz};
  for (int iz = 0; iz < nz; ++iz)
    for (int iy = 0; iy < ny; ++iy)
      for (int ix = 0; ix < nx; ++ix) {
        int i = (iz * ny + iy) * nx + ix, c[3] = {ix, iy, iz};
        m->vol[i] = h[0] * h[1] * h[2];
        for (int d = 0; d < 3; ++d) m->org[3 * i + d] = box[2 * d] + (c[d] + 0.5) * h[d];
        for (int a = 0; a < 9; ++a) { m->Jm[9 * i + a] = 0.0; m->Ji[9 * i + a] = 0.0; }
        for (int d = 0; d < 3; ++d) { m->Jm[9 * i + 4 * d] = 0.5 * h[d]; m->Ji[9 * i + 4 * d] = 2.0 / h[d]; }
        for (int k = 0; k < 6; ++k) {
          int d = k / 2, cc[3] = {c[0], c[1], c[2]};
          double* n = m->nrm + 3 * (6 * i + k);
          n[0] = n[1] = n[2] = 0.0;
          n[d] = (k % 2 ? 1.0 : -1.0) * m->vol[i] / h[d];
          m->nbk[6 * i + k] = k ^ 1;
          cc[d] += k % 2 ? 1 : -1;
          if (cc[d] < 0 || cc[d] >= n3[d]) {
            if (bc[k] == B3_PERIODIC) cc[d] = (cc[d] + n3[d]) % n3[d];
            else { m->nbr[6 * i + k] = -1 - bc[k]; continue; }
          }
          m->nbr[6 * i + k] = (cc[2] * ny + cc[1]) * nx + cc[0];
        }
      }
  mesh3_faces(m);
  return m;
}

static int cmp3(const void* a, const void* b) {
  const long long* x = a; const long long* y = b;
  for (int c = 0; c < 3; ++c) if (x[c] != y[c]) return x[c] < y[c] ? -1 : 1;
  return 0;
}

orc3_mesh* orc3_mesh_tets(int nv, const double* xyz, int nt, const int* tets, const int* vid, const int* fbc) {
  if (nt < 1 || nv < 4) return NULL;
  orc3_mesh* m = mesh3_alloc(KIND3_TET, nt);
  m->canon = malloc(sizeof(int) * 12 * nt);
  /* records (sorted ids of face, cell * 4 + face) for matching */
  long long* rec = malloc(sizeof(long long) * 4 * 4 * nt);
  for (int i = 0; i < nt; ++i) {
    const int* v = tets + 4 * i;
    for (int a = 0; a < 4; ++a)
      if (v[a] < 0 || v[a] >= nv) { free(rec); orc3_mesh_free(m); return NULL; }
    const double *x0 = xyz + 3 * v[0];
    double* J = m->Jm + 9 * i;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) J[3 * a + b] = xyz[3 * v[b + 1] + a] - x0[a];
    double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
    if (!(det > 0.0)) { free(rec); orc3_mesh_free(m); return NULL; }
    m->vol[i] = det / 6.0;
    double* K = m->Ji + 9 * i;   /* inverse by cofactors */
    K[0] = (J[4] * J[8] - J[5] * J[7]) / det; K[1] = (J[2] * J[7] - J[1] * J[8]) / det; K[2] = (J[1] * J[5] - J[2] * J[4]) / det;
    K[3] = (J[5] * J[6] - J[3] * J[8]) / det; K[4] = (J[0] * J[8] - J[2] * J[6]) / det; K[5] = (J[2] * J[3] - J[0] * J[5]) / det;
    K[6] = (J[3] * J[7] - J[4] * J[6]) / det; K[7] = (J[1] * J[6] - J[0] * J[7]) / det; K[8] = (J[0] * J[4] - J[1] * J[3]) / det;
    for (int d = 0; d < 3; ++d) m->org[3 * i + d] = x0[d];
    for (int k = 0; k < 4; ++k) {
      int lv[3], c = 0;
      for (int a = 0; a < 4; ++a) if (a != k) lv[c++] = a;
      /* canonical order: ascending vertex id */
      for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
          if (vid[v[lv[b]]] < vid[v[lv[a]]]) { int t = lv[a]; lv[a] = lv[b]; lv[b] = t; }
      for (int a = 0; a < 3; ++a) m->canon[12 * i + 3 * k + a] = lv[a];
      const double *pa = xyz + 3 * v[lv[0]], *pb = xyz + 3 * v[lv[1]], *pc = xyz + 3 * v[lv[2]], *po = xyz + 3 * v[k];
      double e1[3], e2[3], n[3];
      for (int d = 0; d < 3; ++d) { e1[d] = pb[d] - pa[d]; e2[d] = pc[d] - pa[d]; }
      n[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);
      n[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
      n[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
      double side = n[0] * (po[0] - pa[0]) + n[1] * (po[1] - pa[1]) + n[2] * (po[2] - pa[2]);
      double sg = side > 0.0 ? -1.0 : 1.0;
      for (int d = 0; d < 3; ++d) m->nrm[3 * (4 * i + k) + d] = sg * n[d];
      long long* r = rec + 4 * (4 * i + k);
      r[0] = vid[v[lv[0]]]; r[1] = vid[v[lv[1]]]; r[2] = vid[v[lv[2]]]; r[3] = 4 * i + k;
    }
  }
  qsort(rec, (size_t)4 * nt, sizeof(long long) * 4, cmp3);
  for (int i = 0; i < 4 * nt; ++i) { int c = (int)rec[4 * i + 3]; m->nbr[c] = -1 - B3_TRANSPARENT; m->nbk[c] = -1; }
  for (int i = 0; i < 4 * nt;) {
    int j = i + 1;
    while (j < 4 * nt && cmp3(rec + 4 * i, rec + 4 * j) == 0) ++j;
    if (j - i == 2) {
      int a = (int)rec[4 * i + 3], b = (int)rec[4 * i + 7];
      m->nbr[a] = b / 4; m->nbk[a] = b % 4;
      m->nbr[b] = a / 4; m->nbk[b] = a % 4;
    } else if (j - i == 1) {
      int a = (int)rec[4 * i + 3];
      m->nbr[a] = -1 - (fbc ? fbc[a] : B3_TRANSPARENT);
    } else {
      free(rec); orc3_mesh_free(m); return NULL;   /* a face shared by more than two cells */
    }
    i = j;
  }
  free(rec);
  mesh3_faces(m);
  return m;
}

void orc3_mesh_free(orc3_mesh* m) {
  if (!m) return;
  free(m->vol); free(m->org); free(m->Jm); free(m->Ji); free(m->nrm); free(m->nbr); free(m->nbk);
  free(m->canon); free(m->f_i); free(m->f_k); free(m->f_j); free(m->face_of); free(m->eps);
  free(m);
}

int orc3_mesh_num_elements(const orc3_mesh* m) { return m->N; }
int orc3_mesh_faces_per_element(const orc3_mesh* m) { return m->E; }

/* reference -> physical: x = org + Jm r */
static void to_phys(const orc3_mesh* m, int i, const double* r, double* x) {
  const double *o = m->org + 3 * i, *J = m->Jm + 9 * i;
  for (int a = 0; a < 3; ++a) x[a] = o[a] + J[3 * a] * r[0] + J[3 * a + 1] * r[1] + J[3 * a + 2] * r[2];
}

void orc3_mesh_geometry(const orc3_mesh* m, double* vol, double* cx, double* cy, double* cz) {
  for (int i = 0; i < m->N; ++i) {
    double rc[3], x[3];
    if (m->kind == KIND3_HEX) { rc[0] = rc[1] = rc[2] = 0.0; }
    else { rc[0] = rc[1] = rc[2] = 0.25; }
    to_phys(m, i, rc, x);
    if (vol) vol[i] = m->vol[i];
    if (cx) cx[i] = x[0];
    if (cy) cy[i] = x[1];
    if (cz) cz[i] = x[2];
  }
}

/* ------------------------------------------------------------------ */
/* Solver tables                                                       */
/* ------------------------------------------------------------------ */
struct orc3_solver {
  const orc3_mesh* m;
  int kind, deg, ML, E, NQ, NF, NPT, NPJ;
  double gamma, eps0, alpha0;
  int shock_limiter, llf_global;
  double qw[MAXQ3], fw2[MAXF3];                        /* interior / face weights, each summing to 1 */
  double px[MAXPTS3], py[MAXPTS3], pz[MAXPTS3];        /* reference points (tetrahedra: interior only) */
  double phi[MAXPTS3][MAXML3];                         /* basis there */
  double dref[MAXQ3][3][MAXML3];                       /* reference gradient at the interior points */
  double* fphi;   /* tetrahedra: [N][4][NF][ML] basis at each cell's face points (canonical order) */
  double* fref;   /* tetrahedra: [N][4][NF][3] their reference coordinates */
  double jx[MAXPJ3], jy[MAXPJ3], jz[MAXPJ3], jw[MAXPJ3], jphi[MAXPJ3][MAXML3];
  double *V, *tq, *tqt, *tqtt, *tF;   /* V[N][ML][5]; traces [N][E][NF][5], tF [N][E][NF][3][5] */
  double *fstar, *flxw, *flxf;        /* per face: [nf][NF][5], [nf][5], [nf][5] */
  double* prop;                       /* [N][E] */
  double last_dt;
};

static const double TREF3[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

orc3_solver* orc3_solver_new(const orc3_mesh* m, int deg, double gamma) {
  if (deg < 1 || deg > 3) return NULL;
  orc3_solver* s = calloc(1, sizeof(orc3_solver));
  s->m = m; s->kind = m->kind; s->deg = deg; s->gamma = gamma; s->E = m->E;
  s->eps0 = 1e-12; s->alpha0 = 500.0; s->shock_limiter = 1;
  s->ML = orc3_num_modes(deg);
  int n = deg + 1, E = m->E;
  double Ct[MAXML3][MAXML3];   /* tetrahedra: basis coefficients */
  double g[8], gw[8];
  orc_gauss_legendre(n, g, gw);
  const size_t cap = (size_t)(MAXPJ3 > MAXPTS3 ? MAXPJ3 : MAXPTS3) * MAXML3;
  double *ph = malloc(sizeof(double) * cap), *dx = malloc(sizeof(double) * cap);
  double *dy = malloc(sizeof(double) * cap), *dz = malloc(sizeof(double) * cap);
  if (s->kind == KIND3_HEX) {
    s->NQ = n * n * n; s->NF = n * n;
    for (int c = 0; c < n; ++c)
      for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
          int k = (c * n + b) * n + a;
          s->px[k] = g[a]; s->py[k] = g[b]; s->pz[k] = g[c];
          s->qw[k] = gw[a] * gw[b] * gw[c] / 8.0;
        }
    for (int t = 0; t < n; ++t)
      for (int u = 0; u < n; ++u) s->fw2[t * n + u] = gw[u] * gw[t] / 4.0;
    for (int k = 0; k < 6; ++k) {
      int d = k / 2, d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;   /* tangential directions, x-y-z order */
      double side = k % 2 ? 1.0 : -1.0;
      for (int t = 0; t < n; ++t)
        for (int u = 0; u < n; ++u) {
          int idx = s->NQ + k * s->NF + t * n + u;
          double r[3];
          r[d] = side; r[d1] = g[u]; r[d2] = g[t];
          s->px[idx] = r[0]; s->py[idx] = r[1]; s->pz[idx] = r[2];
        }
    }
    s->NPT = s->NQ + 6 * s->NF;
    orc3_basis_eval(deg, s->NPT, s->px, s->py, s->pz, ph, dx, dy, dz);
  } else {
    tet_basis_coeffs(deg, Ct);   /* once per solver: the Gram-Schmidt runs in long double */
    s->NQ = tet_rule(n, s->px, s->py, s->pz, s->qw);
    double fa[MAXF3], fb[MAXF3];
    s->NF = tri_rule(n, fa, fb, s->fw2);
    s->NPT = s->NQ + 4 * s->NF;
    tet_basis_apply(deg, Ct, s->NQ, s->px, s->py, s->pz, ph, dx, dy, dz);
    /* face points of every cell, from its face's vertices in id order */
    size_t N = (size_t)m->N, NF = (size_t)s->NF, ML = (size_t)s->ML;
    s->fref = malloc(sizeof(double) * N * 4 * NF * 3);
    s->fphi = malloc(sizeof(double) * N * 4 * NF * ML);
    for (size_t i = 0; i < N; ++i)
      for (int k = 0; k < 4; ++k) {
        const int* cv = m->canon + 12 * i + 3 * k;
        double rr[MAXF3], rs[MAXF3], rt[MAXF3];
        for (size_t p = 0; p < NF; ++p) {
          double l1 = fa[p], l2 = fb[p], l0 = 1.0 - l1 - l2;
          double r[3];
          for (int d = 0; d < 3; ++d) r[d] = l0 * TREF3[cv[0]][d] + l1 * TREF3[cv[1]][d] + l2 * TREF3[cv[2]][d];
          rr[p] = r[0]; rs[p] = r[1]; rt[p] = r[2];
          for (int d = 0; d < 3; ++d) s->fref[((i * 4 + k) * NF + p) * 3 + d] = r[d];
        }
        double fp[MAXF3 * MAXML3];
        tet_basis_apply(deg, Ct, (int)NF, rr, rs, rt, fp, NULL, NULL, NULL);
        memcpy(s->fphi + (i * 4 + k) * NF * ML, fp, sizeof(double) * NF * ML);
      }
  }
  int nint = s->kind == KIND3_HEX ? s->NPT : s->NQ;
  for (int p = 0; p < nint; ++p)
    for (int l = 0; l < s->ML; ++l) s->phi[p][l] = ph[p * s->ML + l];
  for (int p = 0; p < s->NQ; ++p)
    for (int l = 0; l < s->ML; ++l) {
      s->dref[p][0][l] = dx[p * s->ML + l];
      s->dref[p][1][l] = dy[p * s->ML + l];
      s->dref[p][2][l] = dz[p * s->ML + l];
    }
  /* projection rule: deg + 3 points per direction */
  int nj = deg + 3;
  if (s->kind == KIND3_HEX) {
    double gj[8], gjw[8];
    orc_gauss_legendre(nj, gj, gjw);
    s->NPJ = nj * nj * nj;
    for (int c = 0; c < nj; ++c)
      for (int b = 0; b < nj; ++b)
        for (int a = 0; a < nj; ++a) {
          int k = (c * nj + b) * nj + a;
          s->jx[k] = gj[a]; s->jy[k] = gj[b]; s->jz[k] = gj[c];
          s->jw[k] = gjw[a] * gjw[b] * gjw[c] / 8.0;
        }
    orc3_basis_eval(deg, s->NPJ, s->jx, s->jy, s->jz, ph, NULL, NULL, NULL);
  } else {
    s->NPJ = tet_rule(nj, s->jx, s->jy, s->jz, s->jw);
    tet_basis_apply(deg, Ct, s->NPJ, s->jx, s->jy, s->jz, ph, NULL, NULL, NULL);
  }
  for (int p = 0; p < s->NPJ; ++p)
    for (int l = 0; l < s->ML; ++l) s->jphi[p][l] = ph[p * s->ML + l];
  free(ph); free(dx); free(dy); free(dz);
  size_t N = (size_t)m->N, NF = (size_t)s->NF, nf = (size_t)m->nfaces;
  s->V = malloc(sizeof(double) * N * s->ML * NV3);
  s->tq = malloc(sizeof(double) * N * E * NF * NV3);
  s->tqt = malloc(sizeof(double) * N * E * NF * NV3);
  s->tqtt = malloc(sizeof(double) * N * E * NF * NV3);
  s->tF = malloc(sizeof(double) * N * E * NF * 3 * NV3);
  s->fstar = malloc(sizeof(double) * nf * NF * NV3);
  s->flxw = malloc(sizeof(double) * nf * NV3);
  s->flxf = malloc(sizeof(double) * nf * NV3);
  s->prop = malloc(sizeof(double) * N * E);
  return s;
}

void orc3_solver_free(orc3_solver* s) {
  if (!s) return;
  free(s->fphi); free(s->fref);
  free(s->V); free(s->tq); free(s->tqt); free(s->tqtt); free(s->tF);
  free(s->fstar); free(s->flxw); free(s->flxf); free(s->prop);
  free(s);
}

void orc3_solver_set_params(orc3_solver* s, double eps0, double alpha0, int shock_limiter) {
  s->eps0 = eps0; s->alpha0 = alpha0; s->shock_limiter = shock_limiter;
}
void orc3_solver_set_llf_global(orc3_solver* s, int flag) { s->llf_global = flag; }
int orc3_solver_num_modes(const orc3_solver* s) { return s->ML; }
int orc3_solver_num_points(const orc3_solver* s) { return s->NPT; }
int orc3_projection_num_points(const orc3_solver* s) { return s->NPJ; }

/* basis at point p of cell i: interior points (and the hexahedra's face
 * points) from the shared table, the tetrahedra's face points per cell */
static const double* phi_at(const orc3_solver* s, int i, int p) {
  if (p < s->NQ || s->kind == KIND3_HEX) return s->phi[p];
  int k = (p - s->NQ) / s->NF, pe = (p - s->NQ) % s->NF;
  return s->fphi + (((size_t)i * 4 + k) * s->NF + pe) * s->ML;
}

static void ref_at(const orc3_solver* s, int i, int p, double* r) {
  if (p < s->NQ || s->kind == KIND3_HEX) { r[0] = s->px[p]; r[1] = s->py[p]; r[2] = s->pz[p]; return; }
  int k = (p - s->NQ) / s->NF, pe = (p - s->NQ) % s->NF;
  const double* f = s->fref + (((size_t)i * 4 + k) * s->NF + pe) * 3;
  r[0] = f[0]; r[1] = f[1]; r[2] = f[2];
}

void orc3_projection_points(const orc3_solver* s, double* xyz) {
  for (int i = 0; i < s->m->N; ++i)
    for (int p = 0; p < s->NPJ; ++p) {
      double r[3] = {s->jx[p], s->jy[p], s->jz[p]};
      to_phys(s->m, i, r, xyz + ((size_t)i * s->NPJ + p) * 3);
    }
}

void orc3_projection_weights(const orc3_solver* s, double* w) {
  for (int p = 0; p < s->NPJ; ++p) w[p] = s->jw[p];
}

void orc3_project(const orc3_solver* s, const double* prim, double* Q) {
  int ML = s->ML;
  double g = s->gamma;
  for (int i = 0; i < s->m->N; ++i) {
    double* Qi = Q + (size_t)i * NV3 * ML;
    for (int c = 0; c < NV3 * ML; ++c) Qi[c] = 0.0;
    for (int p = 0; p < s->NPJ; ++p) {
      const double* w = prim + ((size_t)i * s->NPJ + p) * 5;
      double q[5] = {w[0], w[0] * w[1], w[0] * w[2], w[0] * w[3],
                     w[4] / (g - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3])};
      for (int v = 0; v < NV3; ++v)
        for (int l = 0; l < ML; ++l) Qi[v * ML + l] += s->jw[p] * q[v] * s->jphi[p][l];
    }
  }
}

static void eval_point3(const orc3_solver* s, const double* Qi, const double* phi, double* q) {
  for (int v = 0; v < NV3; ++v) {
    double a = 0.0;
    for (int l = 0; l < s->ML; ++l) a += Qi[v * s->ML + l] * phi[l];
    q[v] = a;
  }
}

void orc3_eval_projection_points(const orc3_solver* s, const double* Q, double* q) {
  for (int i = 0; i < s->m->N; ++i)
    for (int p = 0; p < s->NPJ; ++p)
      eval_point3(s, Q + (size_t)i * NV3 * s->ML, s->jphi[p], q + ((size_t)i * s->NPJ + p) * 5);
}

void orc3_limiter_points(const orc3_solver* s, double* xyz) {
  for (int i = 0; i < s->m->N; ++i)
    for (int p = 0; p < s->NPT; ++p) {
      double r[3];
      ref_at(s, i, p, r);
      to_phys(s->m, i, r, xyz + ((size_t)i * s->NPT + p) * 3);
    }
}

void orc3_eval_limiter_points(const orc3_solver* s, const double* Q, double* q) {
  for (int i = 0; i < s->m->N; ++i)
    for (int p = 0; p < s->NPT; ++p)
      eval_point3(s, Q + (size_t)i * NV3 * s->ML, phi_at(s, i, p), q + ((size_t)i * s->NPT + p) * 5);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.1: moment limiter (Steps 0-2) on one element                 */
/* ------------------------------------------------------------------ */
static double moment_limit3(const orc3_solver* s, int i, double* Qi, int* status) {
  int ML = s->ML;
  double g = s->gamma;
  double qbar[5];
  for (int v = 0; v < NV3; ++v) qbar[v] = Qi[v * ML];
  /* Step 0: non-positive averages are flattened and reported */
  double pbar = qbar[0] > 0.0 ? pressure3(g, qbar) : -1.0;
  if (!(qbar[0] > 0.0) || !(pbar > 0.0)) {
    *status |= ST3_NONPOSITIVE;
    for (int v = 0; v < NV3; ++v)
      for (int l = 1; l < ML; ++l) Qi[v * ML + l] = 0.0;
    return 0.0;
  }
  double dev[MAXPTS3][5];
  for (int p = 0; p < s->NPT; ++p) {
    const double* ph = phi_at(s, i, p);
    for (int v = 0; v < NV3; ++v) {
      double a = 0.0;
      for (int l = 1; l < ML; ++l) a += Qi[v * ML + l] * ph[l];
      dev[p][v] = a;
    }
  }
  /* Step 1: largest theta_rho keeping every point density at eps_rho or above */
  double eps_r = fmin(s->eps0, 0.5 * qbar[0]);
  double th_r = 1.0;
  for (int p = 0; p < s->NPT; ++p) {
    double rm = qbar[0] + dev[p][0];
    if (rm < eps_r) {
      double t = (qbar[0] - eps_r) / (qbar[0] - rm);
      if (t < th_r) th_r = t;
    }
  }
  /* Step 2 (Lemma 1): secant through (0, pbar) and (theta_rho, p of the point) */
  double eps_p = fmin(s->eps0, 0.5 * pbar);
  double th = th_r;
  for (int p = 0; p < s->NPT; ++p) {
    double qt[5];
    for (int v = 0; v < NV3; ++v) qt[v] = qbar[v] + th_r * dev[p][v];
    double pt = pressure3(g, qt);
    if (pt < eps_p) {
      double t = th_r * (pbar - eps_p) / (pbar - pt);
      if (t < th) th = t;
    }
  }
  if (th < 0.0) th = 0.0;
  if (th < 1.0)
    for (int v = 0; v < NV3; ++v)
      for (int l = 1; l < ML; ++l) Qi[v * ML + l] *= th;
  return th;
}

double orc3_moment_limit(const orc3_solver* s, double* Q, double* theta, int* status) {
  int st = 0;
  double mn = 1.0;
#pragma omp parallel for reduction(| : st) reduction(min : mn) schedule(static)
  for (int i = 0; i < s->m->N; ++i) {
    int sti = 0;
    double t = moment_limit3(s, i, Q + (size_t)i * NV3 * s->ML, &sti);
    if (theta) theta[i] = t;
    st |= sti;
    if (t < mn) mn = t;
  }
  if (status) *status |= st;
  return mn;
}

double orc3_wave_speed(const orc3_solver* s, const double* Q) {
  double smax = 0.0;
#pragma omp parallel for reduction(max : smax) schedule(static)
  for (int i = 0; i < s->m->N; ++i) {
    const double* Qi = Q + (size_t)i * NV3 * s->ML;
    double qbar[5];
    for (int v = 0; v < NV3; ++v) qbar[v] = Qi[v * s->ML];
    double a = wave_speed3(s->gamma, qbar);
    if (a > smax) smax = a;
    for (int p = 0; p < s->NPT; ++p) {
      double q[5];
      eval_point3(s, Qi, phi_at(s, i, p), q);
      double b = wave_speed3(s->gamma, q);
      if (b > smax) smax = b;
    }
  }
  return smax;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2-2.3: CK time-averaged flux on one element.  Project F onto  */
/* the basis (interior rule); q_t = -div F^h at the interior points,     */
/* projected onto the modes (it lies in the space) and evaluated at     */
/* every point; F_t = F'(q) q_t, projected; q_tt = -div F_t^h likewise;  */
/* F_tt = F''(q)(q_t, q_t) + F'(q) q_tt; F_T = F + dt/2 F_t + dt^2/6     */
/* F_tt; volume integral Int grad phi . F_T.                             */
/* ------------------------------------------------------------------ */
typedef double pt5[5];
typedef double pt35[3][5];

/* modes of -div of the projection of a flux field given at the interior points */
static void neg_div_modes(const orc3_solver* s, const double* Ji, pt35* Fk, double (*out)[5]) {
  int ML = s->ML, NQ = s->NQ;
  double Fh[MAXML3][3][5];
  for (int l = 0; l < ML; ++l)
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < NV3; ++v) {
        double a = 0.0;
        for (int k = 0; k < NQ; ++k) a += s->qw[k] * Fk[k][d][v] * s->phi[k][l];
        Fh[l][d][v] = a;
      }
  for (int l = 0; l < ML; ++l)
    for (int v = 0; v < NV3; ++v) out[l][v] = 0.0;
  for (int k = 0; k < NQ; ++k) {
    /* physical gradient: d phi / d x_d = sum_a (d r_a / d x_d) d phi / d r_a */
    double div[5] = {0, 0, 0, 0, 0};
    for (int m = 0; m < ML; ++m)
      for (int d = 0; d < 3; ++d) {
        double gd = Ji[0 * 3 + d] * s->dref[k][0][m] + Ji[1 * 3 + d] * s->dref[k][1][m] + Ji[2 * 3 + d] * s->dref[k][2][m];
        for (int v = 0; v < NV3; ++v) div[v] += Fh[m][d][v] * gd;
      }
    for (int l = 0; l < ML; ++l)
      for (int v = 0; v < NV3; ++v) out[l][v] -= s->qw[k] * div[v] * s->phi[k][l];
  }
}

static void ck3(const orc3_solver* s, int i, const double* Qi, double dt, pt5* q, pt5* qt, pt5* qtt, pt35* FT,
                double (*V)[5]) {
  const orc3_mesh* m = s->m;
  int ML = s->ML, NQ = s->NQ, NPT = s->NPT;
  double g = s->gamma;
  const double* Ji = m->Ji + 9 * i;
  pt35* F = malloc(sizeof(pt35) * MAXPTS3);
  pt35* Ft = malloc(sizeof(pt35) * MAXPTS3);
  for (int p = 0; p < NPT; ++p) {
    eval_point3(s, Qi, phi_at(s, i, p), q[p]);
    orc3_flux(g, q[p], &F[p][0][0]);
  }
  double Qt[MAXML3][5], Qtt[MAXML3][5];
  neg_div_modes(s, Ji, F, Qt);
  for (int p = 0; p < NPT; ++p) {
    const double* ph = phi_at(s, i, p);
    for (int v = 0; v < NV3; ++v) {
      double a = 0.0;
      for (int l = 0; l < ML; ++l) a += Qt[l][v] * ph[l];
      qt[p][v] = a;
    }
    double qs[2][5], Fs[2][3][5];
    for (int v = 0; v < NV3; ++v) { qs[0][v] = q[p][v]; qs[1][v] = qt[p][v]; }
    orc3_flux_series(g, 1, &qs[0][0], &Fs[0][0][0]);
    memcpy(Ft[p], Fs[1], sizeof(pt35));
  }
  neg_div_modes(s, Ji, Ft, Qtt);
  for (int p = 0; p < NPT; ++p) {
    const double* ph = phi_at(s, i, p);
    for (int v = 0; v < NV3; ++v) {
      double a = 0.0;
      for (int l = 0; l < ML; ++l) a += Qtt[l][v] * ph[l];
      qtt[p][v] = a;
    }
    /* F_tt = twice the t^2 coefficient of F(q + t q_t + t^2 q_tt / 2) */
    double qs[3][5], Fs[3][3][5];
    for (int v = 0; v < NV3; ++v) { qs[0][v] = q[p][v]; qs[1][v] = qt[p][v]; qs[2][v] = 0.5 * qtt[p][v]; }
    orc3_flux_series(g, 2, &qs[0][0], &Fs[0][0][0]);
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < NV3; ++v)
        FT[p][d][v] = F[p][d][v] + dt / 2.0 * Ft[p][d][v] + dt * dt / 6.0 * 2.0 * Fs[2][d][v];
  }
  /* interior integral of grad phi_l . F_T over the cell */
  for (int l = 0; l < ML; ++l)
    for (int v = 0; v < NV3; ++v) {
      double a = 0.0;
      for (int k = 0; k < NQ; ++k)
        for (int d = 0; d < 3; ++d) {
          double gd = Ji[0 * 3 + d] * s->dref[k][0][l] + Ji[1 * 3 + d] * s->dref[k][1][l] + Ji[2 * 3 + d] * s->dref[k][2][l];
          a += s->qw[k] * gd * FT[k][d][v];
        }
      V[l][v] = m->vol[i] * a;
    }
  free(F); free(Ft);
}

void orc3_ck_element(const orc3_solver* s, const double* Q, int i, double dt, double* q, double* qt,
                     double* qtt, double* FT, double* V) {
  pt5* a = malloc(sizeof(pt5) * MAXPTS3);
  pt5* b = malloc(sizeof(pt5) * MAXPTS3);
  pt5* c = malloc(sizeof(pt5) * MAXPTS3);
  pt35* f = malloc(sizeof(pt35) * MAXPTS3);
  double vv[MAXML3][5];
  ck3(s, i, Q + (size_t)i * NV3 * s->ML, dt, a, b, c, f, vv);
  for (int p = 0; p < s->NPT; ++p)
    for (int v = 0; v < NV3; ++v) {
      if (q) q[p * 5 + v] = a[p][v];
      if (qt) qt[p * 5 + v] = b[p][v];
      if (qtt) qtt[p * 5 + v] = c[p][v];
      if (FT)
        for (int d = 0; d < 3; ++d) FT[(p * 3 + d) * 5 + v] = f[p][d][v];
    }
  if (V)
    for (int l = 0; l < s->ML; ++l)
      for (int v = 0; v < NV3; ++v) V[l * 5 + v] = vv[l][v];
  free(a); free(b); free(c); free(f);
}

/* Sec. 2.4 on a face of unit normal nh: reflective mirrors the momentum,
 * transparent copies; the same map applies to q, q_t and q_tt. */
static void boundary_state3(int bc, const double* nh, const double* qin, double* qout) {
  for (int v = 0; v < NV3; ++v) qout[v] = qin[v];
  if (bc == B3_REFLECT) {
    double mn = qin[1] * nh[0] + qin[2] * nh[1] + qin[3] * nh[2];
    for (int d = 0; d < 3; ++d) qout[1 + d] = qin[1 + d] - 2.0 * mn * nh[d];
  }
}

/* F_T at one point from q, q_t, q_tt (boundary states) */
static void ft_point3(double g, double dt, const double* q, const double* qt, const double* qtt, double* FT) {
  double qs[3][5], Fs[3][3][5];
  for (int v = 0; v < NV3; ++v) { qs[0][v] = q[v]; qs[1][v] = qt[v]; qs[2][v] = 0.5 * qtt[v]; }
  orc3_flux_series(g, 2, &qs[0][0], &Fs[0][0][0]);
  /* F = c0, F_t = c1, F_tt = 2 c2 */
  for (int d = 0; d < 3; ++d)
    for (int v = 0; v < NV3; ++v)
      FT[d * 5 + v] = Fs[0][d][v] + dt / 2.0 * Fs[1][d][v] + dt * dt / 6.0 * 2.0 * Fs[2][d][v];
}

/* ------------------------------------------------------------------ */
/* Sec. 3.3 Step 5(b): largest mu in [0,1] keeping the average pressure */
/* of mu q^c + (1-mu) q^LxF at eps_p = min(eps0, p^LxF/2) or above       */
/* (rho E - |m|^2/2 - kappa rho is quadratic in mu).                     */
/* ------------------------------------------------------------------ */
double orc3_mu_solve(double g, double eps0, const double* ql, const double* qc) {
  double pl = pressure3(g, ql);
  if (!(ql[0] > 0.0) || !(pl > 0.0)) return 0.0;
  double eps_p = fmin(eps0, 0.5 * pl);
  double kappa = eps_p / (g - 1.0);
  double d[5];
  for (int v = 0; v < NV3; ++v) d[v] = qc[v] - ql[v];
  double h0 = ql[0] * ql[4] - 0.5 * (ql[1] * ql[1] + ql[2] * ql[2] + ql[3] * ql[3]) - kappa * ql[0];
  double h1 = ql[0] * d[4] + d[0] * ql[4] - (ql[1] * d[1] + ql[2] * d[2] + ql[3] * d[3]) - kappa * d[0];
  double h2 = d[0] * d[4] - 0.5 * (d[1] * d[1] + d[2] * d[2] + d[3] * d[3]);
  if (qc[0] > 0.0 && h0 + h1 + h2 >= 0.0) return 1.0;
  double disc = h1 * h1 - 4.0 * h0 * h2;
  if (disc < 0.0) disc = 0.0;
  double den = -h1 + sqrt(disc);
  if (!(den > 0.0)) return 0.0;
  double mu = 2.0 * h0 / den;
  if (mu > 1.0) mu = 1.0;
  if (mu < 0.0) mu = 0.0;
  return mu;
}

/* Sec. 3.3 Steps 4-5 with E faces (E <= 6): the negative density flux
 * differences share Lambda = (Gamma^rho - |K| eps_rho/dt) / |their sum|,
 * then mu over every corner of the box of the E proposals. */
int orc3_flux_limit_cell(double g, double eps0, int E, double T, double dt, const double* qbar,
                         const double* fWp, const double* fFp, double* prop) {
  const double(*fW)[5] = (const double(*)[5])fWp;
  const double(*fF)[5] = (const double(*)[5])fFp;
  double Gam[5];
  for (int v = 0; v < NV3; ++v) {
    double a = T / dt * qbar[v];
    for (int k = 0; k < E; ++k) a -= fF[k][v];
    Gam[v] = a;
  }
  double negsum = 0.0;
  int nneg = 0;
  for (int k = 0; k < E; ++k) {
    double df = fF[k][0] - fW[k][0];
    if (df < 0.0) { negsum += df; ++nneg; }
  }
  double eps_r = fmin(eps0, 0.5 * dt / T * Gam[0]);
  if (eps_r < 0.0) eps_r = 0.0;
  double lneg = 1.0;
  if (nneg > 0) {
    lneg = (Gam[0] - T / dt * eps_r) / fabs(negsum);
    if (lneg > 1.0) lneg = 1.0;
    if (lneg < 0.0) lneg = 0.0;
  }
  double Lam[6];
  for (int k = 0; k < E; ++k) Lam[k] = fF[k][0] - fW[k][0] < 0.0 ? lneg : 1.0;
  double qlxf[5];
  for (int v = 0; v < NV3; ++v) {
    double a = 0.0;
    for (int k = 0; k < E; ++k) a += fF[k][v];
    qlxf[v] = qbar[v] - dt / T * a;
  }
  double mmin[6];
  for (int k = 0; k < E; ++k) mmin[k] = 1.0;
  for (int c = 1; c < (1 << E); ++c) {
    double qc[5];
    for (int v = 0; v < NV3; ++v) {
      double a = 0.0;
      for (int k = 0; k < E; ++k) {
        double al = (c >> k) & 1 ? Lam[k] : 0.0;
        a += al * fW[k][v] + (1.0 - al) * fF[k][v];
      }
      qc[v] = qbar[v] - dt / T * a;
    }
    double mu = orc3_mu_solve(g, eps0, qlxf, qc);
    for (int k = 0; k < E; ++k)
      if ((c >> k) & 1 && mu < mmin[k]) mmin[k] = mu;
  }
  for (int k = 0; k < E; ++k) prop[k] = Lam[k] * mmin[k];
  return Gam[0] < 0.0;
}


/* ------------------------------------------------------------------ */
/* Sec. 4.1: shock limiter on (rho, u, v, w, p) (reading G14 in 3D)     */
/* ------------------------------------------------------------------ */
static void primitive3(double g, const double* q, double* w) {
  w[0] = q[0]; w[1] = q[1] / q[0]; w[2] = q[2] / q[0]; w[3] = q[3] / q[0]; w[4] = pressure3(g, q);
}

static void unit_normal(const orc3_mesh* m, int i, int k, double* nh, double* ln) {
  const double* n = m->nrm + 3 * ((size_t)m->E * i + k);
  double l = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int d = 0; d < 3; ++d) nh[d] = n[d] / l;
  if (ln) *ln = l;
}

static double shock_theta3(const orc3_solver* s, const double* Q, int i) {
  const orc3_mesh* m = s->m;
  int ML = s->ML, E = m->E;
  double g = s->gamma;
  const double* Qi = Q + (size_t)i * NV3 * ML;
  double qbar[5];
  for (int v = 0; v < NV3; ++v) qbar[v] = Qi[v * ML];
  if (!(qbar[0] > 0.0)) return 0.0;
  double wbar[5];
  primitive3(g, qbar, wbar);
  double alpha = s->alpha0 * pow(cbrt(m->vol[i]), 1.5);
  double Mx[5], Mn[5];
  for (int c = 0; c < 5; ++c) { Mx[c] = wbar[c] + alpha; Mn[c] = wbar[c] - alpha; }
  for (int k = 0; k < E; ++k) {
    int j = m->nbr[E * i + k];
    double qj[5];
    if (j >= 0) {
      for (int v = 0; v < NV3; ++v) qj[v] = Q[(size_t)j * NV3 * ML + v * ML];
    } else {
      double nh[3];
      unit_normal(m, i, k, nh, NULL);
      boundary_state3(-1 - j, nh, qbar, qj);
    }
    if (!(qj[0] > 0.0)) continue;
    double wj[5];
    primitive3(g, qj, wj);
    for (int c = 0; c < 5; ++c) {
      if (wj[c] > Mx[c]) Mx[c] = wj[c];
      if (wj[c] < Mn[c]) Mn[c] = wj[c];
    }
  }
  double hmax[5], hmin[5];
  for (int c = 0; c < 5; ++c) { hmax[c] = -1e300; hmin[c] = 1e300; }
  for (int p = 0; p < s->NPT; ++p) {
    double q[5], w[5];
    eval_point3(s, Qi, phi_at(s, i, p), q);
    if (!(q[0] > 0.0)) return 0.0;
    primitive3(g, q, w);
    for (int c = 0; c < 5; ++c) {
      if (w[c] > hmax[c]) hmax[c] = w[c];
      if (w[c] < hmin[c]) hmin[c] = w[c];
    }
  }
  double th = 1.0;
  for (int c = 0; c < 5; ++c) {
    if (hmax[c] > wbar[c]) { double t = (Mx[c] - wbar[c]) / (hmax[c] - wbar[c]); if (t < th) th = t; }
    if (hmin[c] < wbar[c]) { double t = (wbar[c] - Mn[c]) / (wbar[c] - hmin[c]); if (t < th) th = t; }
  }
  if (th < 0.0) th = 0.0;
  return th;
}

void orc3_shock_limit(const orc3_solver* s, double* Q, double* theta) {
  int N = s->m->N, ML = s->ML;
  double* th = malloc(sizeof(double) * (size_t)N);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < N; ++i) th[i] = shock_theta3(s, Q, i);
  for (int i = 0; i < N; ++i) {
    if (th[i] < 1.0)
      for (int v = 0; v < NV3; ++v)
        for (int l = 1; l < ML; ++l) Q[(size_t)i * NV3 * ML + v * ML + l] *= th[i];
    if (theta) theta[i] = th[i];
  }
  free(th);
}

/* ------------------------------------------------------------------ */
/* One time step: Sec. 3.3 Steps 1-6 on the faces, then the shock       */
/* limiter (outline Step 5).                                            */
/* ------------------------------------------------------------------ */
int orc3_step(orc3_solver* s, double* Q, double dt_in, double cfl, double* diag, double* theta_mom,
              double* theta_sc, double* theta_face) {
  const orc3_mesh* m = s->m;
  int N = m->N, ML = s->ML, NF = s->NF, NQ = s->NQ, nf = m->nfaces, E = m->E;
  double g = s->gamma;
  int status = 0;

  /* Step 1: moment limiter */
  int nmom = 0;
  {
    int st = 0;
#pragma omp parallel for reduction(| : st) reduction(+ : nmom) schedule(static)
    for (int i = 0; i < N; ++i) {
      int sti = 0;
      double t = moment_limit3(s, i, Q + (size_t)i * NV3 * ML, &sti);
      if (theta_mom) theta_mom[i] = t;
      if (t < 1.0) ++nmom;
      st |= sti;
    }
    status |= st;
  }
  double sw = orc3_wave_speed(s, Q);
  double dt = dt_in > 0.0 ? dt_in : cfl * m->hmin / sw;
  s->last_dt = dt;

  /* Step 2: time-averaged fluxes, volume integrals, face traces */
#pragma omp parallel for schedule(static)
  for (int i = 0; i < N; ++i) {
    pt5* q = malloc(sizeof(pt5) * MAXPTS3);
    pt5* qt = malloc(sizeof(pt5) * MAXPTS3);
    pt5* qtt = malloc(sizeof(pt5) * MAXPTS3);
    pt35* FT = malloc(sizeof(pt35) * MAXPTS3);
    double V[MAXML3][5];
    ck3(s, i, Q + (size_t)i * NV3 * ML, dt, q, qt, qtt, FT, V);
    for (int l = 0; l < ML; ++l)
      for (int v = 0; v < NV3; ++v) s->V[((size_t)i * ML + l) * NV3 + v] = V[l][v];
    for (int k = 0; k < E; ++k)
      for (int p = 0; p < NF; ++p) {
        size_t t = (((size_t)i * E + k) * NF + p) * NV3;
        int src = NQ + k * NF + p;
        for (int v = 0; v < NV3; ++v) {
          s->tq[t + v] = q[src][v]; s->tqt[t + v] = qt[src][v]; s->tqtt[t + v] = qtt[src][v];
          for (int d = 0; d < 3; ++d) s->tF[t * 3 + d * NV3 + v] = FT[src][d][v];
        }
      }
    free(q); free(qt); free(qtt); free(FT);
  }

  /* Step 3 (face loop): LLF flux at the face points, f^LxW, f^LxF */
#pragma omp parallel for schedule(static)
  for (int f = 0; f < nf; ++f) {
    int i = m->f_i[f], ki = m->f_k[f], j = m->f_j[f];
    int kj = j >= 0 ? m->nbk[E * i + ki] : -1;
    const double* n = m->nrm + 3 * ((size_t)E * i + ki);   /* outward for i, scaled by the face area */
    double nh[3], ln;
    unit_normal(m, i, ki, nh, &ln);
    double fw[5] = {0, 0, 0, 0, 0};
    for (int p = 0; p < NF; ++p) {
      size_t ti = (((size_t)i * E + ki) * NF + p) * NV3;
      const double* qm = s->tq + ti;
      const double* Fm = s->tF + ti * 3;
      double qp[5], Fp[15];
      if (j >= 0) {
        /* both cells see the face's points in the same order */
        size_t tj = (((size_t)j * E + kj) * NF + p) * NV3;
        for (int v = 0; v < NV3; ++v) qp[v] = s->tq[tj + v];
        for (int c = 0; c < 15; ++c) Fp[c] = s->tF[tj * 3 + c];
      } else {
        double qtp[5], qttp[5];
        boundary_state3(-1 - j, nh, qm, qp);
        boundary_state3(-1 - j, nh, s->tqt + ti, qtp);
        boundary_state3(-1 - j, nh, s->tqtt + ti, qttp);
        ft_point3(g, dt, qp, qtp, qttp, Fp);
      }
      double sp = sw;
      if (!s->llf_global) {
        double am = wave_speed3(g, qm), ap = wave_speed3(g, qp);
        double a = am > ap ? am : ap;
        if (a < sp) sp = a;
      }
      double* fs = s->fstar + ((size_t)f * NF + p) * NV3;
      for (int v = 0; v < NV3; ++v) {
        /* Eq. LLF times the face area */
        double fn = 0.0;
        for (int d = 0; d < 3; ++d) fn += n[d] * (Fp[d * 5 + v] + Fm[d * 5 + v]);
        fs[v] = 0.5 * fn - 0.5 * sp * ln * (qp[v] - qm[v]);
        fw[v] += s->fw2[p] * fs[v];
      }
    }
    /* Lax-Friedrichs flux of the cell averages (Sec. 3.2) */
    double qi[5], qj[5];
    for (int v = 0; v < NV3; ++v) qi[v] = Q[(size_t)i * NV3 * ML + v * ML];
    if (j >= 0) {
      for (int v = 0; v < NV3; ++v) qj[v] = Q[(size_t)j * NV3 * ML + v * ML];
    } else {
      boundary_state3(-1 - j, nh, qi, qj);
    }
    double Fi[15], Fj[15];
    orc3_flux(g, qi, Fi);
    orc3_flux(g, qj, Fj);
    for (int v = 0; v < NV3; ++v) {
      double fn = 0.0;
      for (int d = 0; d < 3; ++d) fn += n[d] * (Fj[d * 5 + v] + Fi[d * 5 + v]);
      s->flxw[(size_t)f * NV3 + v] = fw[v];
      s->flxf[(size_t)f * NV3 + v] = 0.5 * fn - 0.5 * ln * sw * (qj[v] - qi[v]);
    }
  }

  /* Steps 4-5: Lambda proposals per element face */
  int cfl_bad = 0;
#pragma omp parallel for reduction(| : cfl_bad) schedule(static)
  for (int i = 0; i < N; ++i) {
    double qbar[5], fW[6][5], fF[6][5];
    for (int v = 0; v < NV3; ++v) qbar[v] = Q[(size_t)i * NV3 * ML + v * ML];
    for (int k = 0; k < E; ++k) {
      int f = m->face_of[E * i + k];
      double ek = m->eps[E * i + k];
      for (int v = 0; v < NV3; ++v) {
        fW[k][v] = ek * s->flxw[(size_t)f * NV3 + v];
        fF[k][v] = ek * s->flxf[(size_t)f * NV3 + v];
      }
    }
    if (orc3_flux_limit_cell(g, s->eps0, E, m->vol[i], dt, qbar, &fW[0][0], &fF[0][0], s->prop + (size_t)i * E))
      cfl_bad = 1;
  }
  if (cfl_bad) status |= ST3_CFL;

  /* Step 6: theta per face (min of both sides) and the update */
  int nface_lim = 0;
  double* Qn = malloc(sizeof(double) * (size_t)N * NV3 * ML);
#pragma omp parallel for reduction(+ : nface_lim) schedule(static)
  for (int i = 0; i < N; ++i) {
    const double* Qi = Q + (size_t)i * NV3 * ML;
    double* Qo = Qn + (size_t)i * NV3 * ML;
    double vol = m->vol[i];
    double Eint[MAXML3][5];
    for (int l = 0; l < ML; ++l) for (int v = 0; v < NV3; ++v) Eint[l][v] = 0.0;
    double avg_upd[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < E; ++k) {
      int f = m->face_of[E * i + k];
      double ek = m->eps[E * i + k];
      int j = m->nbr[E * i + k];
      double th = s->prop[(size_t)i * E + k];
      if (j >= 0) { double o = s->prop[(size_t)j * E + m->nbk[E * i + k]]; if (o < th) th = o; }
      if (theta_face) theta_face[(size_t)i * E + k] = th;
      if (th < 1.0 && ek > 0) ++nface_lim;
      for (int v = 0; v < NV3; ++v)
        avg_upd[v] += ek * (th * s->flxw[(size_t)f * NV3 + v] + (1.0 - th) * s->flxf[(size_t)f * NV3 + v]);
      /* face integral of phi_l F*.n over this face */
      for (int p = 0; p < NF; ++p) {
        const double* fs = s->fstar + ((size_t)f * NF + p) * NV3;
        const double* ph = phi_at(s, i, NQ + k * NF + p);
        for (int l = 0; l < ML; ++l)
          for (int v = 0; v < NV3; ++v) Eint[l][v] += s->fw2[p] * ph[l] * ek * fs[v];
      }
    }
    for (int v = 0; v < NV3; ++v) {
      Qo[v * ML] = Qi[v * ML] - dt / vol * avg_upd[v];
      for (int l = 1; l < ML; ++l)
        Qo[v * ML + l] = Qi[v * ML + l] + dt / vol * (s->V[((size_t)i * ML + l) * NV3 + v] - Eint[l][v]);
    }
  }
  memcpy(Q, Qn, sizeof(double) * (size_t)N * NV3 * ML);
  free(Qn);

  /* shock limiter on the new state */
  int nsc = 0;
  if (s->shock_limiter) {
    double* th = theta_sc ? theta_sc : malloc(sizeof(double) * (size_t)N);
    orc3_shock_limit(s, Q, th);
    for (int i = 0; i < N; ++i) if (th[i] < 1.0) ++nsc;
    if (!theta_sc) free(th);
  } else if (theta_sc) {
    for (int i = 0; i < N; ++i) theta_sc[i] = 1.0;
  }

  if (diag) {
    double mr = 1e300, mp = 1e300, tot[5] = {0, 0, 0, 0, 0};
    for (int i = 0; i < N; ++i) {
      const double* Qi = Q + (size_t)i * NV3 * ML;
      double qb[5];
      for (int v = 0; v < NV3; ++v) qb[v] = Qi[v * ML];
      double pb = pressure3(g, qb);
      if (qb[0] < mr) mr = qb[0];
      if (pb < mp) mp = pb;
      for (int v = 0; v < NV3; ++v) tot[v] += m->vol[i] * qb[v];
      for (int v = 0; v < NV3; ++v) if (!isfinite(qb[v])) status |= ST3_NAN;
    }
    for (int c = 0; c < ORC3_DIAG_LEN; ++c) diag[c] = 0.0;
    diag[ORC3_D_S] = sw; diag[ORC3_D_DT] = dt; diag[ORC3_D_MINRHO] = mr; diag[ORC3_D_MINP] = mp;
    diag[ORC3_D_MASS] = tot[0]; diag[ORC3_D_MOMX] = tot[1]; diag[ORC3_D_MOMY] = tot[2];
    diag[ORC3_D_MOMZ] = tot[3]; diag[ORC3_D_ENERGY] = tot[4]; diag[ORC3_D_NMOM] = nmom;
    diag[ORC3_D_NFACE] = nface_lim; diag[ORC3_D_NSC] = nsc; diag[ORC3_D_STATUS] = status;
  }
  return status;
}

double orc3_last_fluxes(const orc3_solver* s, double* fw, double* ff) {
  const orc3_mesh* m = s->m;
  int E = m->E;
  for (int i = 0; i < m->N; ++i)
    for (int k = 0; k < E; ++k) {
      int f = m->face_of[E * i + k];
      double ek = m->eps[E * i + k];
      for (int v = 0; v < NV3; ++v) {
        fw[((size_t)i * E + k) * NV3 + v] = ek * s->flxw[(size_t)f * NV3 + v];
        ff[((size_t)i * E + k) * NV3 + v] = ek * s->flxf[(size_t)f * NV3 + v];
      }
    }
  return s->last_dt;
}
