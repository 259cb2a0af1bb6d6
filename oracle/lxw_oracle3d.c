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
 */
#include "lxw_oracle3d.h"
#include "lxw_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NV3 5
#define MAXML3 20                 /* modes of degree 3 */
#define MAXN3 4                   /* points per direction (degree 3) */
#define MAXQ3 (MAXN3 * MAXN3 * MAXN3)
#define MAXF3 (MAXN3 * MAXN3)
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
/* Cartesian mesh: box cells, six faces each                            */
/* ------------------------------------------------------------------ */
struct orc3_mesh {
  int nx, ny, nz, N;
  double box[6], h[3];
  int bc[6];
  int* nbr;      /* [N][6]: neighbour, or -1 - bc on a boundary side */
  int nfaces;
  int *f_i, *f_k, *f_j;   /* face: owner i, its local face k, neighbour j (or -1 - bc) */
  int* face_of;  /* [N][6] face index */
  double* eps;   /* [N][6] +1 owner side, -1 neighbour side */
  double hmin;
};

orc3_mesh* orc3_mesh_cartesian(int nx, int ny, int nz, const double* box, const int* bc) {
  if (nx < 1 || ny < 1 || nz < 1) return NULL;
  orc3_mesh* m = calloc(1, sizeof(orc3_mesh));
  m->nx = nx; m->ny = ny; m->nz = nz; m->N = nx * ny * nz;
  memcpy(m->box, box, sizeof(double) * 6);
  memcpy(m->bc, bc, sizeof(int) * 6);
  m->h[0] = (box[1] - box[0]) / nx; m->h[1] = (box[3] - box[2]) / ny; m->h[2] = (box[5] - box[4]) / nz;
  int N = m->N, n3[3] = {nx, ny, nz};
  m->nbr = malloc(sizeof(int) * 6 * N);
  for (int iz = 0; iz < nz; ++iz)
    for (int iy = 0; iy < ny; ++iy)
      for (int ix = 0; ix < nx; ++ix) {
        int i = (iz * ny + iy) * nx + ix, c[3] = {ix, iy, iz};
        for (int k = 0; k < 6; ++k) {
          int d = k / 2, step = k % 2 ? 1 : -1;
          int cc[3] = {c[0], c[1], c[2]};
          cc[d] += step;
          int side = k;   /* the domain side this face lies on when cc leaves the box */
          if (cc[d] < 0 || cc[d] >= n3[d]) {
            if (bc[side] == B3_PERIODIC) cc[d] = (cc[d] + n3[d]) % n3[d];
            else { m->nbr[6 * i + k] = -1 - bc[side]; continue; }
          }
          m->nbr[6 * i + k] = (cc[2] * ny + cc[1]) * nx + cc[0];
        }
      }
  /* faces: every + face of a cell, and the - faces on non-periodic boundaries */
  m->f_i = malloc(sizeof(int) * 6 * N); m->f_k = malloc(sizeof(int) * 6 * N); m->f_j = malloc(sizeof(int) * 6 * N);
  m->face_of = malloc(sizeof(int) * 6 * N);
  m->eps = malloc(sizeof(double) * 6 * N);
  int nf = 0;
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < 6; ++k) {
      int j = m->nbr[6 * i + k];
      if (k % 2 == 1 || j < 0) {
        m->f_i[nf] = i; m->f_k[nf] = k; m->f_j[nf] = j;
        m->face_of[6 * i + k] = nf; m->eps[6 * i + k] = 1.0;
        ++nf;
      }
    }
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < 6; k += 2) {
      int j = m->nbr[6 * i + k];
      if (j >= 0) {   /* the - face of i is the + face of j */
        m->face_of[6 * i + k] = m->face_of[6 * j + k + 1];
        m->eps[6 * i + k] = -1.0;
      }
    }
  m->nfaces = nf;
  double vol = m->h[0] * m->h[1] * m->h[2];
  double surf = 2.0 * (m->h[0] * m->h[1] + m->h[1] * m->h[2] + m->h[0] * m->h[2]);
  m->hmin = 3.0 * vol / surf;
  return m;
}

void orc3_mesh_free(orc3_mesh* m) {
  if (!m) return;
  free(m->nbr); free(m->f_i); free(m->f_k); free(m->f_j); free(m->face_of); free(m->eps);
  free(m);
}

int orc3_mesh_num_elements(const orc3_mesh* m) { return m->N; }

static void cell_origin(const orc3_mesh* m, int i, double* o) {
  int ix = i % m->nx, iy = (i / m->nx) % m->ny, iz = i / (m->nx * m->ny);
  o[0] = m->box[0] + (ix + 0.5) * m->h[0];
  o[1] = m->box[2] + (iy + 0.5) * m->h[1];
  o[2] = m->box[4] + (iz + 0.5) * m->h[2];
}

void orc3_mesh_geometry(const orc3_mesh* m, double* vol, double* cx, double* cy, double* cz) {
  for (int i = 0; i < m->N; ++i) {
    double o[3];
    cell_origin(m, i, o);
    if (vol) vol[i] = m->h[0] * m->h[1] * m->h[2];
    if (cx) cx[i] = o[0];
    if (cy) cy[i] = o[1];
    if (cz) cz[i] = o[2];
  }
}

/* outward normal of face k scaled by the face area */
static void face_normal(const orc3_mesh* m, int k, double* n) {
  int d = k / 2;
  double area = m->h[0] * m->h[1] * m->h[2] / m->h[d];
  n[0] = n[1] = n[2] = 0.0;
  n[d] = k % 2 ? area : -area;
}

/* ------------------------------------------------------------------ */
/* Solver tables                                                       */
/* ------------------------------------------------------------------ */
struct orc3_solver {
  const orc3_mesh* m;
  int deg, ML, n, NQ, NF, NPT, NPJ;
  double gamma, eps0, alpha0;
  int shock_limiter, llf_global;
  double qw[MAXQ3], fw2[MAXF3];                     /* interior / face weights, each summing to 1 */
  double px[MAXPTS3], py[MAXPTS3], pz[MAXPTS3];     /* reference points */
  double phi[MAXPTS3][MAXML3], dxi[MAXPTS3][MAXML3], deta[MAXPTS3][MAXML3], dzeta[MAXPTS3][MAXML3];
  double jx[MAXPJ3], jy[MAXPJ3], jz[MAXPJ3], jw[MAXPJ3], jphi[MAXPJ3][MAXML3];
  double *V, *tq, *tqt, *tqtt, *tF;   /* V[N][ML][5]; traces [N][6][NF][5], tF [N][6][NF][3][5] */
  double *fstar, *flxw, *flxf;        /* per face: [nf][NF][5], [nf][5], [nf][5] */
  double* prop;                       /* [N][6] */
  double last_dt;
};

orc3_solver* orc3_solver_new(const orc3_mesh* m, int deg, double gamma) {
  if (deg < 1 || deg > 3) return NULL;
  orc3_solver* s = calloc(1, sizeof(orc3_solver));
  s->m = m; s->deg = deg; s->gamma = gamma;
  s->eps0 = 1e-12; s->alpha0 = 500.0; s->shock_limiter = 1;
  s->ML = orc3_num_modes(deg);
  int n = deg + 1;
  s->n = n;
  double g[8], gw[8];
  orc_gauss_legendre(n, g, gw);
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
  /* the projection rule has more points than the limiter set */
  const size_t cap = (size_t)(MAXPJ3 > MAXPTS3 ? MAXPJ3 : MAXPTS3) * MAXML3;
  double *ph = malloc(sizeof(double) * cap), *dx = malloc(sizeof(double) * cap);
  double *dy = malloc(sizeof(double) * cap), *dz = malloc(sizeof(double) * cap);
  orc3_basis_eval(deg, s->NPT, s->px, s->py, s->pz, ph, dx, dy, dz);
  for (int p = 0; p < s->NPT; ++p)
    for (int l = 0; l < s->ML; ++l) {
      s->phi[p][l] = ph[p * s->ML + l];
      s->dxi[p][l] = dx[p * s->ML + l];
      s->deta[p][l] = dy[p * s->ML + l];
      s->dzeta[p][l] = dz[p * s->ML + l];
    }
  /* projection rule: deg + 3 points per direction */
  int nj = deg + 3;
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
  for (int p = 0; p < s->NPJ; ++p)
    for (int l = 0; l < s->ML; ++l) s->jphi[p][l] = ph[p * s->ML + l];
  free(ph); free(dx); free(dy); free(dz);
  size_t N = (size_t)m->N, NF = (size_t)s->NF, nf = (size_t)m->nfaces;
  s->V = malloc(sizeof(double) * N * s->ML * NV3);
  s->tq = malloc(sizeof(double) * N * 6 * NF * NV3);
  s->tqt = malloc(sizeof(double) * N * 6 * NF * NV3);
  s->tqtt = malloc(sizeof(double) * N * 6 * NF * NV3);
  s->tF = malloc(sizeof(double) * N * 6 * NF * 3 * NV3);
  s->fstar = malloc(sizeof(double) * nf * NF * NV3);
  s->flxw = malloc(sizeof(double) * nf * NV3);
  s->flxf = malloc(sizeof(double) * nf * NV3);
  s->prop = malloc(sizeof(double) * N * 6);
  return s;
}

void orc3_solver_free(orc3_solver* s) {
  if (!s) return;
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

void orc3_projection_points(const orc3_solver* s, double* xyz) {
  const orc3_mesh* m = s->m;
  for (int i = 0; i < m->N; ++i) {
    double o[3];
    cell_origin(m, i, o);
    for (int p = 0; p < s->NPJ; ++p) {
      double* r = xyz + ((size_t)i * s->NPJ + p) * 3;
      r[0] = o[0] + 0.5 * m->h[0] * s->jx[p];
      r[1] = o[1] + 0.5 * m->h[1] * s->jy[p];
      r[2] = o[2] + 0.5 * m->h[2] * s->jz[p];
    }
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
  const orc3_mesh* m = s->m;
  for (int i = 0; i < m->N; ++i) {
    double o[3];
    cell_origin(m, i, o);
    for (int p = 0; p < s->NPT; ++p) {
      double* r = xyz + ((size_t)i * s->NPT + p) * 3;
      r[0] = o[0] + 0.5 * m->h[0] * s->px[p];
      r[1] = o[1] + 0.5 * m->h[1] * s->py[p];
      r[2] = o[2] + 0.5 * m->h[2] * s->pz[p];
    }
  }
}

void orc3_eval_limiter_points(const orc3_solver* s, const double* Q, double* q) {
  for (int i = 0; i < s->m->N; ++i)
    for (int p = 0; p < s->NPT; ++p)
      eval_point3(s, Q + (size_t)i * NV3 * s->ML, s->phi[p], q + ((size_t)i * s->NPT + p) * 5);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.1: moment limiter (Steps 0-2) on one element                 */
/* ------------------------------------------------------------------ */
static double moment_limit3(const orc3_solver* s, double* Qi, int* status) {
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
  for (int p = 0; p < s->NPT; ++p)
    for (int v = 0; v < NV3; ++v) {
      double a = 0.0;
      for (int l = 1; l < ML; ++l) a += Qi[v * ML + l] * s->phi[p][l];
      dev[p][v] = a;
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
    double t = moment_limit3(s, Q + (size_t)i * NV3 * s->ML, &sti);
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
      eval_point3(s, Qi, s->phi[p], q);
      double b = wave_speed3(s->gamma, q);
      if (b > smax) smax = b;
    }
  }
  return smax;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2-2.3: CK time-averaged flux on one element.  Project F onto  */
/* the basis (interior rule), q_t = -div F^h, F_t = F'(q) q_t; project,  */
/* q_tt = -div F_t^h, F_tt = F''(q)(q_t, q_t) + F'(q) q_tt;              */
/* F_T = F + dt/2 F_t + dt^2/6 F_tt; volume integral Int grad phi . F_T. */
/* ------------------------------------------------------------------ */
typedef double pt5[5];
typedef double pt35[3][5];

static void ck3(const orc3_solver* s, const double* Qi, double dt, pt5* q, pt5* qt, pt5* qtt, pt35* FT,
                double (*V)[5]) {
  const orc3_mesh* m = s->m;
  int ML = s->ML, NQ = s->NQ, NPT = s->NPT;
  double g = s->gamma;
  double sc[3] = {2.0 / m->h[0], 2.0 / m->h[1], 2.0 / m->h[2]};
  double vol = m->h[0] * m->h[1] * m->h[2];
  /* physical gradients of the basis: grad phi = (2/hx d/dxi, 2/hy d/deta, 2/hz d/dzeta) */
  double (*gb)[3][MAXML3] = malloc(sizeof(double) * MAXPTS3 * 3 * MAXML3);
  for (int p = 0; p < NPT; ++p)
    for (int l = 0; l < ML; ++l) {
      gb[p][0][l] = sc[0] * s->dxi[p][l];
      gb[p][1][l] = sc[1] * s->deta[p][l];
      gb[p][2][l] = sc[2] * s->dzeta[p][l];
    }
  pt35* F = malloc(sizeof(pt35) * MAXPTS3);
  pt35* Ft = malloc(sizeof(pt35) * MAXPTS3);
  pt35* Ftt = malloc(sizeof(pt35) * MAXPTS3);
  for (int p = 0; p < NPT; ++p) {
    eval_point3(s, Qi, s->phi[p], q[p]);
    orc3_flux(g, q[p], &F[p][0][0]);
  }
  /* Galerkin expansion of F (the three directions) */
  double Fh[MAXML3][3][5];
  for (int l = 0; l < ML; ++l)
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < NV3; ++v) {
        double a = 0.0;
        for (int k = 0; k < NQ; ++k) a += s->qw[k] * F[k][d][v] * s->phi[k][l];
        Fh[l][d][v] = a;
      }
  /* q_t = -div F^h and F_t = F'(q) q_t at every point */
  for (int p = 0; p < NPT; ++p) {
    for (int v = 0; v < NV3; ++v) {
      double a = 0.0;
      for (int l = 0; l < ML; ++l)
        for (int d = 0; d < 3; ++d) a += Fh[l][d][v] * gb[p][d][l];
      qt[p][v] = -a;
    }
    double qs[2][5], Fs[2][3][5];
    for (int v = 0; v < NV3; ++v) { qs[0][v] = q[p][v]; qs[1][v] = qt[p][v]; }
    orc3_flux_series(g, 1, &qs[0][0], &Fs[0][0][0]);
    memcpy(Ft[p], Fs[1], sizeof(pt35));
  }
  double Fth[MAXML3][3][5];
  for (int l = 0; l < ML; ++l)
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < NV3; ++v) {
        double a = 0.0;
        for (int k = 0; k < NQ; ++k) a += s->qw[k] * Ft[k][d][v] * s->phi[k][l];
        Fth[l][d][v] = a;
      }
  /* q_tt = -div F_t^h; F_tt = twice the t^2 coefficient of F(q + t q_t + t^2 q_tt / 2) */
  for (int p = 0; p < NPT; ++p) {
    for (int v = 0; v < NV3; ++v) {
      double a = 0.0;
      for (int l = 0; l < ML; ++l)
        for (int d = 0; d < 3; ++d) a += Fth[l][d][v] * gb[p][d][l];
      qtt[p][v] = -a;
    }
    double qs[3][5], Fs[3][3][5];
    for (int v = 0; v < NV3; ++v) { qs[0][v] = q[p][v]; qs[1][v] = qt[p][v]; qs[2][v] = 0.5 * qtt[p][v]; }
    orc3_flux_series(g, 2, &qs[0][0], &Fs[0][0][0]);
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < NV3; ++v) Ftt[p][d][v] = 2.0 * Fs[2][d][v];
  }
  for (int p = 0; p < NPT; ++p)
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < NV3; ++v)
        FT[p][d][v] = F[p][d][v] + dt / 2.0 * Ft[p][d][v] + dt * dt / 6.0 * Ftt[p][d][v];
  /* interior integral of grad phi_l . F_T over the cell */
  for (int l = 0; l < ML; ++l)
    for (int v = 0; v < NV3; ++v) {
      double a = 0.0;
      for (int k = 0; k < NQ; ++k)
        for (int d = 0; d < 3; ++d) a += s->qw[k] * gb[k][d][l] * FT[k][d][v];
      V[l][v] = vol * a;
    }
  free(gb); free(F); free(Ft); free(Ftt);
}

void orc3_ck_element(const orc3_solver* s, const double* Q, int i, double dt, double* q, double* qt,
                     double* qtt, double* FT, double* V) {
  pt5* a = malloc(sizeof(pt5) * MAXPTS3);
  pt5* b = malloc(sizeof(pt5) * MAXPTS3);
  pt5* c = malloc(sizeof(pt5) * MAXPTS3);
  pt35* f = malloc(sizeof(pt35) * MAXPTS3);
  double vv[MAXML3][5];
  ck3(s, Q + (size_t)i * NV3 * s->ML, dt, a, b, c, f, vv);
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

/* ------------------------------------------------------------------ */
/* Sec. 2.4 on a face of axis d: reflective flips the normal momentum,  */
/* transparent copies; the same map applies to q, q_t and q_tt.          */
/* ------------------------------------------------------------------ */
static void boundary_state3(int bc, int d, const double* qin, double* qout) {
  for (int v = 0; v < NV3; ++v) qout[v] = qin[v];
  if (bc == B3_REFLECT) qout[1 + d] = -qin[1 + d];
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

static double shock_theta3(const orc3_solver* s, const double* Q, int i) {
  const orc3_mesh* m = s->m;
  int ML = s->ML;
  double g = s->gamma;
  const double* Qi = Q + (size_t)i * NV3 * ML;
  double qbar[5];
  for (int v = 0; v < NV3; ++v) qbar[v] = Qi[v * ML];
  if (!(qbar[0] > 0.0)) return 0.0;
  double wbar[5];
  primitive3(g, qbar, wbar);
  double alpha = s->alpha0 * pow(cbrt(m->h[0] * m->h[1] * m->h[2]), 1.5);
  double Mx[5], Mn[5];
  for (int c = 0; c < 5; ++c) { Mx[c] = wbar[c] + alpha; Mn[c] = wbar[c] - alpha; }
  for (int k = 0; k < 6; ++k) {
    int j = m->nbr[6 * i + k];
    double qj[5];
    if (j >= 0) {
      for (int v = 0; v < NV3; ++v) qj[v] = Q[(size_t)j * NV3 * ML + v * ML];
    } else {
      boundary_state3(-1 - j, k / 2, qbar, qj);
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
    eval_point3(s, Qi, s->phi[p], q);
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
/* One time step: Sec. 3.3 Steps 1-6 on six faces, then the shock      */
/* limiter (outline Step 5).                                            */
/* ------------------------------------------------------------------ */
int orc3_step(orc3_solver* s, double* Q, double dt_in, double cfl, double* diag, double* theta_mom,
              double* theta_sc, double* theta_face) {
  const orc3_mesh* m = s->m;
  int N = m->N, ML = s->ML, NF = s->NF, NQ = s->NQ, nf = m->nfaces;
  double g = s->gamma;
  double vol = m->h[0] * m->h[1] * m->h[2];
  int status = 0;

  /* Step 1: moment limiter */
  int nmom = 0;
  {
    int st = 0;
#pragma omp parallel for reduction(| : st) reduction(+ : nmom) schedule(static)
    for (int i = 0; i < N; ++i) {
      int sti = 0;
      double t = moment_limit3(s, Q + (size_t)i * NV3 * ML, &sti);
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
    ck3(s, Q + (size_t)i * NV3 * ML, dt, q, qt, qtt, FT, V);
    for (int l = 0; l < ML; ++l)
      for (int v = 0; v < NV3; ++v) s->V[((size_t)i * ML + l) * NV3 + v] = V[l][v];
    for (int k = 0; k < 6; ++k)
      for (int p = 0; p < NF; ++p) {
        size_t t = (((size_t)i * 6 + k) * NF + p) * NV3;
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
    int d = ki / 2, kj = ki ^ 1;   /* the neighbour's matching face */
    double n[3];
    face_normal(m, ki, n);   /* outward for i, scaled by the face area */
    double ln = fabs(n[d]);
    double fw[5] = {0, 0, 0, 0, 0};
    for (int p = 0; p < NF; ++p) {
      size_t ti = (((size_t)i * 6 + ki) * NF + p) * NV3;
      const double* qm = s->tq + ti;
      const double* Fm = s->tF + ti * 3;
      double qp[5], Fp[15];
      if (j >= 0) {
        /* both cells see the face's points in the same order */
        size_t tj = (((size_t)j * 6 + kj) * NF + p) * NV3;
        for (int v = 0; v < NV3; ++v) qp[v] = s->tq[tj + v];
        for (int c = 0; c < 15; ++c) Fp[c] = s->tF[tj * 3 + c];
      } else {
        double qtp[5], qttp[5];
        boundary_state3(-1 - j, d, qm, qp);
        boundary_state3(-1 - j, d, s->tqt + ti, qtp);
        boundary_state3(-1 - j, d, s->tqtt + ti, qttp);
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
        fs[v] = 0.5 * n[d] * (Fp[d * 5 + v] + Fm[d * 5 + v]) - 0.5 * sp * ln * (qp[v] - qm[v]);
        fw[v] += s->fw2[p] * fs[v];
      }
    }
    /* Lax-Friedrichs flux of the cell averages (Sec. 3.2) */
    double qi[5], qj[5];
    for (int v = 0; v < NV3; ++v) qi[v] = Q[(size_t)i * NV3 * ML + v * ML];
    if (j >= 0) {
      for (int v = 0; v < NV3; ++v) qj[v] = Q[(size_t)j * NV3 * ML + v * ML];
    } else {
      boundary_state3(-1 - j, d, qi, qj);
    }
    double Fi[15], Fj[15];
    orc3_flux(g, qi, Fi);
    orc3_flux(g, qj, Fj);
    for (int v = 0; v < NV3; ++v) {
      s->flxw[(size_t)f * NV3 + v] = fw[v];
      s->flxf[(size_t)f * NV3 + v] = 0.5 * n[d] * (Fj[d * 5 + v] + Fi[d * 5 + v]) - 0.5 * ln * sw * (qj[v] - qi[v]);
    }
  }

  /* Steps 4-5: Lambda proposals per element face */
  int cfl_bad = 0;
#pragma omp parallel for reduction(| : cfl_bad) schedule(static)
  for (int i = 0; i < N; ++i) {
    double qbar[5], fW[6][5], fF[6][5];
    for (int v = 0; v < NV3; ++v) qbar[v] = Q[(size_t)i * NV3 * ML + v * ML];
    for (int k = 0; k < 6; ++k) {
      int f = m->face_of[6 * i + k];
      double ek = m->eps[6 * i + k];
      for (int v = 0; v < NV3; ++v) {
        fW[k][v] = ek * s->flxw[(size_t)f * NV3 + v];
        fF[k][v] = ek * s->flxf[(size_t)f * NV3 + v];
      }
    }
    if (orc3_flux_limit_cell(g, s->eps0, 6, vol, dt, qbar, &fW[0][0], &fF[0][0], s->prop + (size_t)i * 6))
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
    double Eint[MAXML3][5];
    for (int l = 0; l < ML; ++l) for (int v = 0; v < NV3; ++v) Eint[l][v] = 0.0;
    double avg_upd[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 6; ++k) {
      int f = m->face_of[6 * i + k];
      double ek = m->eps[6 * i + k];
      int j = m->nbr[6 * i + k];
      double th = s->prop[(size_t)i * 6 + k];
      if (j >= 0) { double o = s->prop[(size_t)j * 6 + (k ^ 1)]; if (o < th) th = o; }
      if (theta_face) theta_face[(size_t)i * 6 + k] = th;
      if (th < 1.0 && ek > 0) ++nface_lim;
      for (int v = 0; v < NV3; ++v)
        avg_upd[v] += ek * (th * s->flxw[(size_t)f * NV3 + v] + (1.0 - th) * s->flxf[(size_t)f * NV3 + v]);
      /* face integral of phi_l F*.n over this face */
      for (int p = 0; p < NF; ++p) {
        const double* fs = s->fstar + ((size_t)f * NF + p) * NV3;
        int pt = NQ + k * NF + p;
        for (int l = 0; l < ML; ++l)
          for (int v = 0; v < NV3; ++v) Eint[l][v] += s->fw2[p] * s->phi[pt][l] * ek * fs[v];
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
      for (int v = 0; v < NV3; ++v) tot[v] += vol * qb[v];
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
  for (int i = 0; i < m->N; ++i)
    for (int k = 0; k < 6; ++k) {
      int f = m->face_of[6 * i + k];
      double ek = m->eps[6 * i + k];
      for (int v = 0; v < NV3; ++v) {
        fw[((size_t)i * 6 + k) * NV3 + v] = ek * s->flxw[(size_t)f * NV3 + v];
        ff[((size_t)i * 6 + k) * NV3 + v] = ek * s->flxf[(size_t)f * NV3 + v];
      }
    }
  return s->last_dt;
}
