/*
 * dgw_oracle.c -- plain, slow, FP64 CPU oracle for the DG wall-model operators.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may include, link or call this file;
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it. It shares no
 * code, header, table generator or helper with the CUDA library.
 *
 * What it computes (Krank, Kronbichler & Wall, arXiv 1705.08813):
 *   - SIPG pressure Laplacian            -L(q,p)             Sec. 4.2, eq. (ipflux)
 *   - velocity divergence                -C(q,u)             Sec. 4.2, velocity divergence item
 *   - Lax-Friedrichs convective term      F^c(v,u)            Sec. 4.2, convective item
 *   - multiscale viscous term            -F^nu(vbar,vtil;u)  Sec. 4.2, eq. (viscous_multiscale),
 *                                                             eq. (harmweights), eq. (minvt)
 *   - eddy viscosity nu_t                                     Sec. 2.2, eq. (mix), (lmix), (ydes)
 *   - enrichment u~ = psi * sum N_B u~_B                      Sec. 3.1, eq. (enrichment)
 *   - wall laws psi(y+): Spalding (inverted by Newton) and van Driest (Appendix A: Table A1
 *     support points + 9-point Gauss rule, eq. (psinum))    Sec. 3.2, eq. (psi)
 *   - CG solve of -L p = b on the zero-mean subspace
 *
 * Every weak form is evaluated literally: loop over cells, over quadrature points, over every
 * test function, with the basis tabulated in full 3-D at each point (no sum factorisation), and
 * over the six faces of each cell with the neighbour state re-evaluated at the same face point.
 * Quadrature rules are the method's own (Sec. 4.4): k+1 Gauss points per direction for linear
 * terms, floor(3k/2)+1 for the convective term, q_w Gauss points in the wall-normal direction of
 * enriched cells; faces take the count of the adjacent enriched cell in the wall-normal
 * tangential direction. "extra_q" adds points in every direction (used by exactness pins only).
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   tau_IP: (k+1)^2 * A(dK)/V(K), interior faces weighted 1/2, boundary faces 1; face value
 *     max of both sides; x10 on no-slip walls for the viscous term (Sec. 4.2 says only "by
 *     Hillewaert"); Spalding B = 5.17; Gauss-Lobatto nodal points; homogeneous Neumann data for
 *     the pressure on walls; enriched wall faces belong to the enriched-face class with the mirror
 *     state; nu_t frozen from a separately passed velocity field.

 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KAPPA 0.41          /* Sec. 3.2 (eq. psi) and eq. (lmix) */
#define APLUS 26.0          /* van Driest damping constant, eq. (lmix) */
#define B_SPALDING 5.17     /* Spalding's additive constant (not given in the paper) */
#define C_DES 0.85          /* eq. (ydes) */
#define BETA_DES 6.0        /* eq. (ydes) */
#define WALL_PENALTY 10.0   /* Sec. 4.2: tau_IP x10 on Dirichlet faces (viscous term) */
#define MAXP 16             /* max points / nodes per direction */

typedef struct {
  int nx, ny, nz;        /* cells per direction */
  int k;                 /* polynomial degree of ubar and p */
  int enrich_l;          /* 0 or 1: degree of the enrichment weights N^l */
  int q_wall;            /* Gauss points in wall-normal direction of enriched cells */
  int geometry;          /* 0 channel (boxes), 1 bump (curved, isoparametric Q_k) */
  int wall_law;          /* 0 Spalding, 1 van Driest */
  int n_layers;          /* enriched cell layers per wall; 0 disables enrichment */
  int extra_q;           /* extra quadrature points per direction (pins only) */
  int full_q;            /* 1: enriched cells take q_wall points in every direction and faces touching
                            them q_wall per tangential direction (the paper's 8^3 rule, Sec. 4.4) */
  double lx, ly, lz;     /* domain lengths; channel walls at y = +-ly/2, bump y in [yw(x), ly] */
  double gamma;          /* tanh grading factor */
  double nu;             /* kinematic viscosity */
  double tau_w;          /* wall shear stress (rho = 1) at every wall node */
} dgo_params;

typedef struct {
  dgo_params P;
  int k, n1, nc, ne, nef;     /* n1 = k+1; nef = (l+1)^3 enriched functions per component */
  long np, nu;                /* pressure and velocity vector lengths */
  double gl[MAXP];            /* Gauss-Lobatto nodes on [0,1] */
  double *xv, *yv, *zv;       /* channel vertex coordinates */
  double *X;                  /* per cell nodal positions [nc][n1^3][3] */
  int *enr, *enr_cell;        /* cell -> enriched index (-1) ; enriched index -> cell */
  double *ywall;              /* per enriched cell: 8 vertex wall distances */
  double *tauv;               /* per enriched cell: 8 vertex wall shear stresses */
  int *tsrc;                  /* per enriched cell: 8 wall-node indices (the node that defines y_B) */
  int *slot;                  /* cell -> enriched index whether switched on or off (-1: not a wall cell) */
  double yp_off;              /* switch-off threshold: a wall column is off if all points have y+ < yp_off */
  double *dye;                /* per cell wall-normal width */
  double *tau_cell;           /* per cell penalty tau_IP */
  unsigned char *active;      /* optional: only these cells' outputs are computed (NULL = all) */
} omesh;

/* ------------------------------------------------------------------------------------------ */
/* 1-D rules                                                                                  */
/* ------------------------------------------------------------------------------------------ */

/* Legendre P_n and P_n' at x in [-1,1] by the three-term recurrence. */
static void legendre(int n, double x, double *p, double *dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int m = 2; m <= n; ++m) {
    double p2 = ((2.0 * m - 1.0) * x * p1 - (m - 1.0) * p0) / m;
    p0 = p1; p1 = p2;
  }
  *p = p1;
  *dp = (fabs(x) < 1.0) ? n * (x * p1 - p0) / (x * x - 1.0) : 0.5 * n * (n + 1) * pow(x, n + 1);
}

/* n-point Gauss-Legendre rule on [0,1] (Newton on the roots of P_n). */
void dgo_gauss(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double t = cos(M_PI * (i + 0.75) / (n + 0.5)), p, dp;
    for (int it = 0; it < 100; ++it) {
      legendre(n, t, &p, &dp);
      double dt = p / dp;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    legendre(n, t, &p, &dp);
    /* ascending order on [0,1] */
    x[n - 1 - i] = 0.5 * (1.0 + t);
    w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dp * dp);   /* 2/((1-t^2)P'^2) scaled by 1/2 */
  }
}

/* n-point Gauss-Lobatto nodes on [0,1]: endpoints and roots of P'_{n-1}. */
void dgo_lobatto(int n, double *x) {
  int m = n - 1;
  x[0] = 0.0; x[n - 1] = 1.0;
  for (int i = 1; i < n - 1; ++i) {
    double t = -cos(M_PI * i / m);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(m, t, &p, &dp);
      double d2p = (2.0 * t * dp - m * (m + 1.0) * p) / (1.0 - t * t);
      double dt = dp / d2p;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 + t);
  }
}

/* Lagrange polynomial i on the nodes, value and derivative at s. */
static void lagrange(int n, const double *nodes, int i, double s, double *v, double *d) {
  double val = 1.0, der = 0.0;
  for (int j = 0; j < n; ++j) {
    if (j == i) continue;
    double f = 1.0 / (nodes[i] - nodes[j]);
    der = der * (s - nodes[j]) * f + val * f;
    val *= (s - nodes[j]) * f;
  }
  *v = val; *d = der;
}

/* ------------------------------------------------------------------------------------------ */
/* Wall laws (Sec. 3.2 and Appendix A)                                                        */
/* ------------------------------------------------------------------------------------------ */

/* Spalding's law y+ = psi + e^{-kB}(e^{k psi} - 1 - k psi - (k psi)^2/2 - (k psi)^3/6), inverted
 * by bracketed Newton. Returns psi, writes d psi / d y+. */
double dgo_psi_spalding(double yp, double *dpsi) {
  const double k = KAPPA, eb = exp(-KAPPA * B_SPALDING);
  if (yp <= 0.0) { if (dpsi) *dpsi = 1.0; return 0.0; }
  double lo = 0.0, hi = yp, x = fmin(yp, B_SPALDING + log1p(yp) / KAPPA);
  for (int it = 0; it < 200; ++it) {
    double kx = k * x, g, gp;
    if (kx > 700.0) { hi = x; x = 0.5 * (lo + hi); continue; }
    double e = exp(kx);
    g = x + eb * (e - 1.0 - kx - 0.5 * kx * kx - kx * kx * kx / 6.0) - yp;
    gp = 1.0 + eb * k * (e - 1.0 - kx - 0.5 * kx * kx);
    if (g > 0.0) hi = x; else lo = x;
    double xn = x - g / gp;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (fabs(xn - x) <= 1e-16 * (1.0 + fabs(x))) { x = xn; break; }
    x = xn;
  }
  if (dpsi) {
    double kx = k * x;
    *dpsi = 1.0 / (1.0 + eb * k * (exp(kx) - 1.0 - kx - 0.5 * kx * kx));
  }
  return x;
}

/* Integrand of van Driest's law, eq. (psi): 2/(1+sqrt(1+(2 k y (1-exp(-y/A)))^2)). */
static double vd_integrand(double y) {
  double a = 2.0 * KAPPA * y * (1.0 - exp(-y / APLUS));
  return 2.0 / (1.0 + sqrt(1.0 + a * a));
}

/* Table A1 support points and values (printed in the paper's Appendix A). */
static const double VD_Y[9] = {0.0, 5.0, 11.0, 24.0, 59.0, 144.0, 361.0, 946.0, 2517.0};
static const double VD_PSI[9] = {0.0, 4.88298776233176, 8.91824406645381, 12.3978516813118,
                                 15.1875389926298, 17.4177125619900, 19.6484300823042,
                                 21.9930107788854, 24.3778307011372};

/* psi_i + integral over [y_i, y] with a 9-point Gauss rule, eq. (psinum). */
double dgo_psi_vd_from(int i, double yp) {
  double x[9], w[9];
  dgo_gauss(9, x, w);
  double a = VD_Y[i], h = yp - a, s = 0.0;
  for (int q = 0; q < 9; ++q) s += w[q] * vd_integrand(a + h * x[q]);
  return VD_PSI[i] + h * s;
}

double dgo_psi_vandriest(double yp, double *dpsi) {
  if (yp <= 0.0) { if (dpsi) *dpsi = 1.0; return 0.0; }
  int i = 0;
  while (i < 8 && VD_Y[i + 1] <= yp) ++i;
  if (dpsi) *dpsi = vd_integrand(yp);   /* d psi/dy+ is the integrand (Appendix A) */
  return dgo_psi_vd_from(i, yp);
}

static double wall_law(const omesh *M, double yp, double *dpsi) {
  return M->P.wall_law == 1 ? dgo_psi_vandriest(yp, dpsi) : dgo_psi_spalding(yp, dpsi);
}

/* ------------------------------------------------------------------------------------------ */
/* Mesh                                                                                       */
/* ------------------------------------------------------------------------------------------ */

static double bump_wall(const dgo_params *P, double x) {
  double xc = 0.5 * P->lx, s = x - xc;
  if (fabs(s) < 1.0) { double c = cos(M_PI * s / 2.0); return 0.3 * c * c; }
  return 0.0;
}

static double grading(double gamma, double eta) {   /* [0,1] -> [-1,1], Sec. 5.1 mapping */
  return tanh(gamma * (2.0 * eta - 1.0)) / tanh(gamma);
}

/* Physical point of the logical coordinates (i + s0, j + s1, kz + s2) of the bump geometry. */
static void bump_map(const dgo_params *P, double a0, double a1, double a2, double *x) {
  double xx = P->lx * a0 / P->nx;
  double yw = bump_wall(P, xx);
  double f = grading(P->gamma, a1 / P->ny);
  x[0] = xx;
  x[1] = yw + (P->ly - yw) * 0.5 * (1.0 + f);
  x[2] = P->lz * a2 / P->nz;
}

static inline int cell_id(const omesh *M, int i, int j, int k) {
  return i + M->P.nx * (j + M->P.ny * k);
}

static void vertex_pos(const omesh *M, int i, int j, int kz, double *x) {
  if (M->P.geometry == 0) { x[0] = M->xv[i]; x[1] = M->yv[j]; x[2] = M->zv[kz]; }
  else bump_map(&M->P, i, j, kz, x);
}

/* Mapping from the nodal positions: x(xi), J = dx/dxi, detJ, Jinv = dxi/dx. */
static void map_point(const omesh *M, int c, const double *xi, double *x, double J[3][3],
                      double *detJ, double Ji[3][3]) {
  int n1 = M->n1;
  double l[3][MAXP], dl[3][MAXP];
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < n1; ++a) lagrange(n1, M->gl, a, xi[d], &l[d][a], &dl[d][a]);
  double xs[3] = {0, 0, 0}, Jm[3][3] = {{0}};
  const double *Xc = M->X + (size_t)c * n1 * n1 * n1 * 3;
  for (int c2 = 0; c2 < n1; ++c2)
    for (int b = 0; b < n1; ++b)
      for (int a = 0; a < n1; ++a) {
        const double *Xn = Xc + 3 * (a + n1 * (b + n1 * c2));
        double v = l[0][a] * l[1][b] * l[2][c2];
        double g0 = dl[0][a] * l[1][b] * l[2][c2];
        double g1 = l[0][a] * dl[1][b] * l[2][c2];
        double g2 = l[0][a] * l[1][b] * dl[2][c2];
        for (int e = 0; e < 3; ++e) {
          xs[e] += v * Xn[e];
          Jm[e][0] += g0 * Xn[e]; Jm[e][1] += g1 * Xn[e]; Jm[e][2] += g2 * Xn[e];
        }
      }
  double det = Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1])
             - Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0])
             + Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
  if (x) for (int e = 0; e < 3; ++e) x[e] = xs[e];
  if (J) memcpy(J, Jm, sizeof(Jm));
  *detJ = det;
  Ji[0][0] = (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1]) / det;
  Ji[0][1] = (Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2]) / det;
  Ji[0][2] = (Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1]) / det;
  Ji[1][0] = (Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2]) / det;
  Ji[1][1] = (Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0]) / det;
  Ji[1][2] = (Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2]) / det;
  Ji[2][0] = (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]) / det;
  Ji[2][1] = (Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1]) / det;
  Ji[2][2] = (Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0]) / det;
}

static int is_enriched_row(const omesh *M, int j) {
  int L = M->P.n_layers;
  return L > 0 && (j < L || j >= M->P.ny - L);
}

/* Surface measure factor of face (dir d) at xi: |cof(J) e_d| and the outward normal for the
 * face xi_d = side (side 0 -> outward normal along -grad xi_d). */
static double face_geom(const double Ji[3][3], double detJ, int d, int side, double *n) {
  double g[3] = {Ji[d][0], Ji[d][1], Ji[d][2]};   /* grad xi_d */
  double nrm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  double s = side ? 1.0 : -1.0;
  for (int e = 0; e < 3; ++e) n[e] = s * g[e] / nrm;
  return fabs(detJ) * nrm;   /* dA = |detJ| |grad xi_d| dxi_t1 dxi_t2 */
}

void *dgo_mesh_create(const dgo_params *P) {
  if (P->k < 1 || P->k + 1 > MAXP - 2 || P->nx < 1 || P->ny < 1 || P->nz < 1) return NULL;
  omesh *M = (omesh *)calloc(1, sizeof(omesh));
  M->P = *P;
  M->k = P->k; M->n1 = P->k + 1;
  M->nc = P->nx * P->ny * P->nz;
  M->nef = P->enrich_l == 0 ? 1 : 8;
  int n1 = M->n1, n3 = n1 * n1 * n1;
  dgo_lobatto(n1, M->gl);
  M->xv = (double *)malloc(sizeof(double) * (P->nx + 1));
  M->yv = (double *)malloc(sizeof(double) * (P->ny + 1));
  M->zv = (double *)malloc(sizeof(double) * (P->nz + 1));
  for (int i = 0; i <= P->nx; ++i) M->xv[i] = P->lx * i / P->nx;
  for (int j = 0; j <= P->ny; ++j) M->yv[j] = 0.5 * P->ly * grading(P->gamma, (double)j / P->ny);
  for (int i = 0; i <= P->nz; ++i) M->zv[i] = P->lz * i / P->nz;
  M->X = (double *)malloc(sizeof(double) * (size_t)M->nc * n3 * 3);
  M->enr = (int *)malloc(sizeof(int) * M->nc);
  M->dye = (double *)malloc(sizeof(double) * M->nc);
  M->tau_cell = (double *)malloc(sizeof(double) * M->nc);
  /* enriched numbering: bottom layer(s) then top layer(s), lexicographic (x fastest, then z) */
  int ne = 0;
  for (int c = 0; c < M->nc; ++c) M->enr[c] = -1;
  for (int pass = 0; pass < 2; ++pass)
    for (int j = 0; j < P->ny; ++j) {
      if (!is_enriched_row(M, j)) continue;
      int bottom = j < P->n_layers && (pass == 0);
      int top = j >= P->ny - P->n_layers && (pass == 1) && !(j < P->n_layers);
      if (!(bottom || top)) continue;
      for (int kz = 0; kz < P->nz; ++kz)
        for (int i = 0; i < P->nx; ++i) M->enr[cell_id(M, i, j, kz)] = ne++;
    }
  M->ne = ne;
  M->enr_cell = (int *)malloc(sizeof(int) * (ne > 0 ? ne : 1));
  for (int c = 0; c < M->nc; ++c) if (M->enr[c] >= 0) M->enr_cell[M->enr[c]] = c;
  /* enr[] is the switched-on view used by every operator; slot[] keeps the DoF layout */
  M->slot = (int *)malloc(sizeof(int) * M->nc);
  memcpy(M->slot, M->enr, sizeof(int) * M->nc);
  M->yp_off = 0.0;
  M->np = (long)M->nc * n3;
  M->nu = 3L * M->np + 3L * M->nef * ne;
  /* nodal positions */
  for (int kz = 0; kz < P->nz; ++kz)
    for (int j = 0; j < P->ny; ++j)
      for (int i = 0; i < P->nx; ++i) {
        int c = cell_id(M, i, j, kz);
        double *Xc = M->X + (size_t)c * n3 * 3;
        for (int cc = 0; cc < n1; ++cc)
          for (int b = 0; b < n1; ++b)
            for (int a = 0; a < n1; ++a) {
              double *Xn = Xc + 3 * (a + n1 * (b + n1 * cc));
              if (P->geometry == 0) {
                Xn[0] = M->xv[i] + (M->xv[i + 1] - M->xv[i]) * M->gl[a];
                Xn[1] = M->yv[j] + (M->yv[j + 1] - M->yv[j]) * M->gl[b];
                Xn[2] = M->zv[kz] + (M->zv[kz + 1] - M->zv[kz]) * M->gl[cc];
              } else {
                bump_map(P, i + M->gl[a], j + M->gl[b], kz + M->gl[cc], Xn);
              }
            }
        /* wall-normal width: mean of the four vertical edge lengths */
        double s = 0.0;
        for (int e = 0; e < 4; ++e) {
          double lo[3], hi[3];
          vertex_pos(M, i + (e & 1), j, kz + (e >> 1), lo);
          vertex_pos(M, i + (e & 1), j + 1, kz + (e >> 1), hi);
          s += sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                    (hi[2] - lo[2]) * (hi[2] - lo[2]));
        }
        M->dye[c] = 0.25 * s;
      }
  /* penalty: tau = (k+1)^2 * A/V, interior faces weighted 1/2, wall faces 1 */
  {
    double gx[MAXP], gw[MAXP];
    int nq = n1 + 1;
    dgo_gauss(nq, gx, gw);
    for (int c = 0; c < M->nc; ++c) {
      int j = (c / P->nx) % P->ny;
      double V = 0.0, A = 0.0;
      for (int q2 = 0; q2 < nq; ++q2)
        for (int q1 = 0; q1 < nq; ++q1)
          for (int q0 = 0; q0 < nq; ++q0) {
            double xi[3] = {gx[q0], gx[q1], gx[q2]}, J[3][3], Ji[3][3], det;
            map_point(M, c, xi, NULL, J, &det, Ji);
            V += fabs(det) * gw[q0] * gw[q1] * gw[q2];
          }
      for (int f = 0; f < 6; ++f) {
        int d = f / 2, side = f % 2, t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
        int wall = (d == 1) && ((side == 0 && j == 0) || (side == 1 && j == P->ny - 1));
        double a = 0.0;
        for (int q2 = 0; q2 < nq; ++q2)
          for (int q1 = 0; q1 < nq; ++q1) {
            double xi[3], n[3], J[3][3], Ji[3][3], det;
            xi[d] = side; xi[t1] = gx[q1]; xi[t2] = gx[q2];
            map_point(M, c, xi, NULL, J, &det, Ji);
            a += face_geom(Ji, det, d, side, n) * gw[q1] * gw[q2];
          }
        A += (wall ? 1.0 : 0.5) * a;
      }
      M->tau_cell[c] = (double)(n1 * n1) * A / V;
    }
  }
  /* vertex wall distances (closest wall node) and wall shear stresses of enriched cells */
  M->ywall = (double *)malloc(sizeof(double) * 8 * (ne > 0 ? ne : 1));
  M->tauv = (double *)malloc(sizeof(double) * 8 * (ne > 0 ? ne : 1));
  M->tsrc = (int *)malloc(sizeof(int) * 8 * (ne > 0 ? ne : 1));
  for (int e = 0; e < ne; ++e) {
    int c = M->enr_cell[e], i = c % P->nx, j = (c / P->nx) % P->ny, kz = c / (P->nx * P->ny);
    for (int v = 0; v < 8; ++v) {
      int vi = i + (v & 1), vj = j + ((v >> 1) & 1), vk = kz + (v >> 2);
      double xv[3];
      vertex_pos(M, vi, vj, vk, xv);
      /* closest wall node B (index wall * nx * nz + i + nx * k, periodic indices) */
      double best = 1e300;
      int src = 0;
      if (P->geometry == 0) {
        double db = xv[1] - M->yv[0], dt = M->yv[P->ny] - xv[1];
        best = fmin(db, dt);
        src = (db <= dt ? 0 : P->nx * P->nz) + vi % P->nx + P->nx * (vk % P->nz);
      } else {
        for (int wk = 0; wk <= P->nz; ++wk)
          for (int wi = 0; wi <= P->nx; ++wi)
            for (int wj = 0; wj <= P->ny; wj += P->ny) {
              double w[3];
              vertex_pos(M, wi, wj, wk, w);
              double d2 = (w[0] - xv[0]) * (w[0] - xv[0]) + (w[1] - xv[1]) * (w[1] - xv[1]) +
                          (w[2] - xv[2]) * (w[2] - xv[2]);
              if (d2 < best) {
                best = d2;
                src = (wj ? P->nx * P->nz : 0) + wi % P->nx + P->nx * (wk % P->nz);
              }
            }
        best = sqrt(best);
      }
      M->ywall[8 * e + v] = best;
      M->tauv[8 * e + v] = P->tau_w;
      M->tsrc[8 * e + v] = src;
    }
  }
  return M;
}

/* Restrict the operators to the outputs of the cells with mask[c] != 0 (mask == NULL: all). */
void dgo_set_active(void *h, const unsigned char *mask) {
  omesh *M = (omesh *)h;
  free(M->active);
  M->active = NULL;
  if (mask) {
    M->active = (unsigned char *)malloc(M->nc);
    memcpy(M->active, mask, M->nc);
  }
}

void dgo_mesh_destroy(void *h) {
  omesh *M = (omesh *)h;
  if (!M) return;
  free(M->active);
  free(M->xv); free(M->yv); free(M->zv); free(M->X); free(M->enr); free(M->enr_cell); free(M->slot);
  free(M->ywall); free(M->tauv); free(M->tsrc); free(M->dye); free(M->tau_cell); free(M);
}

void dgo_mesh_info(void *h, long *np, long *nu, long *ne) {
  omesh *M = (omesh *)h;
  *np = M->np; *nu = M->nu; *ne = M->ne;
}

/* Standard nodal positions [cell][n1^3][3] (x-fastest local index). */
void dgo_node_coords(void *h, double *out) {
  omesh *M = (omesh *)h;
  memcpy(out, M->X, sizeof(double) * (size_t)M->np * 3);
}

void dgo_cell_tau(void *h, double *out) {
  omesh *M = (omesh *)h;
  memcpy(out, M->tau_cell, sizeof(double) * M->nc);
}

/* ------------------------------------------------------------------------------------------ */
/* Point tabulation                                                                           */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
  double x[3], J[3][3], Ji[3][3], detJ;
  int n3;
  double *phi, *gphi;               /* standard basis values and physical gradients */
  int enriched, nef;
  double yh, tauh, yp, psi, dpsi, gyp[3];
  double ephi[8], egphi[8][3];      /* psi N_B and gradients */
} ptab;

static void ptab_alloc(ptab *t, const omesh *M) {
  t->n3 = M->n1 * M->n1 * M->n1;
  t->phi = (double *)malloc(sizeof(double) * t->n3);
  t->gphi = (double *)malloc(sizeof(double) * 3 * t->n3);
}
static void ptab_free(ptab *t) { free(t->phi); free(t->gphi); }

/* Trilinear (or constant for l=0) weights N_B and reference gradients. */
static void q1_basis(int nef, const double *xi, double *N, double gN[][3]) {
  if (nef == 1) { N[0] = 1.0; gN[0][0] = gN[0][1] = gN[0][2] = 0.0; return; }
  for (int v = 0; v < 8; ++v) {
    double f[3], df[3];
    for (int d = 0; d < 3; ++d) {
      int b = (v >> d) & 1;
      f[d] = b ? xi[d] : 1.0 - xi[d];
      df[d] = b ? 1.0 : -1.0;
    }
    N[v] = f[0] * f[1] * f[2];
    gN[v][0] = df[0] * f[1] * f[2];
    gN[v][1] = f[0] * df[1] * f[2];
    gN[v][2] = f[0] * f[1] * df[2];
  }
}

static void tabulate(const omesh *M, int c, const double *xi, ptab *t) {
  int n1 = M->n1;
  map_point(M, c, xi, t->x, t->J, &t->detJ, t->Ji);
  double l[3][MAXP], dl[3][MAXP];
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < n1; ++a) lagrange(n1, M->gl, a, xi[d], &l[d][a], &dl[d][a]);
  for (int cc = 0; cc < n1; ++cc)
    for (int b = 0; b < n1; ++b)
      for (int a = 0; a < n1; ++a) {
        int i = a + n1 * (b + n1 * cc);
        double r[3] = {dl[0][a] * l[1][b] * l[2][cc], l[0][a] * dl[1][b] * l[2][cc],
                       l[0][a] * l[1][b] * dl[2][cc]};
        t->phi[i] = l[0][a] * l[1][b] * l[2][cc];
        for (int e = 0; e < 3; ++e)
          t->gphi[3 * i + e] = r[0] * t->Ji[0][e] + r[1] * t->Ji[1][e] + r[2] * t->Ji[2][e];
      }
  int en = M->enr[c];
  t->enriched = en >= 0;
  t->nef = M->nef;
  if (!t->enriched) return;
  /* Sec. 3.2: y_h and tau_w,h interpolated with the linear C0 functions on the cell's vertices */
  double N8[8], gN8r[8][3], gN8[8][3];
  q1_basis(8, xi, N8, gN8r);
  for (int v = 0; v < 8; ++v)
    for (int e = 0; e < 3; ++e)
      gN8[v][e] = gN8r[v][0] * t->Ji[0][e] + gN8r[v][1] * t->Ji[1][e] + gN8r[v][2] * t->Ji[2][e];
  double yh = 0.0, th = 0.0, gy[3] = {0, 0, 0}, gt[3] = {0, 0, 0};
  for (int v = 0; v < 8; ++v) {
    yh += N8[v] * M->ywall[8 * en + v];
    th += N8[v] * M->tauv[8 * en + v];
    for (int e = 0; e < 3; ++e) {
      gy[e] += gN8[v][e] * M->ywall[8 * en + v];
      gt[e] += gN8[v][e] * M->tauv[8 * en + v];
    }
  }
  double nu = M->P.nu, st = sqrt(th);
  t->yh = yh; t->tauh = th;
  t->yp = yh * st / nu;
  for (int e = 0; e < 3; ++e) t->gyp[e] = (st * gy[e] + yh * gt[e] / (2.0 * st)) / nu;
  t->psi = wall_law(M, t->yp, &t->dpsi);
  /* enrichment functions psi * N_B^l, eq. (enrichment); gradient by the chain rule */
  double Nl[8], gNlr[8][3];
  q1_basis(M->nef, xi, Nl, gNlr);
  for (int v = 0; v < M->nef; ++v) {
    double gNl[3];
    for (int e = 0; e < 3; ++e)
      gNl[e] = gNlr[v][0] * t->Ji[0][e] + gNlr[v][1] * t->Ji[1][e] + gNlr[v][2] * t->Ji[2][e];
    t->ephi[v] = t->psi * Nl[v];
    for (int e = 0; e < 3; ++e) t->egphi[v][e] = t->psi * gNl[e] + Nl[v] * t->dpsi * t->gyp[e];
  }
}

/* Velocity state at a tabulated point: ubar, grad ubar, util, grad util (G[a][b] = d u_a/d x_b). */
typedef struct { double ub[3], gb[3][3], ut[3], gt[3][3]; } vstate;

static void eval_vel(const omesh *M, const double *u, int c, const ptab *t, vstate *s) {
  int n3 = t->n3;
  memset(s, 0, sizeof(*s));
  for (int a = 0; a < 3; ++a) {
    const double *uc = u + ((size_t)c * 3 + a) * n3;
    for (int i = 0; i < n3; ++i) {
      s->ub[a] += t->phi[i] * uc[i];
      for (int e = 0; e < 3; ++e) s->gb[a][e] += t->gphi[3 * i + e] * uc[i];
    }
  }
  if (!t->enriched) return;
  int en = M->enr[c];
  const double *ue = u + 3L * M->np + (size_t)en * 3 * M->nef;
  for (int a = 0; a < 3; ++a)
    for (int v = 0; v < M->nef; ++v) {
      double cv = ue[a * M->nef + v];
      s->ut[a] += t->ephi[v] * cv;
      for (int e = 0; e < 3; ++e) s->gt[a][e] += t->egphi[v][e] * cv;
    }
}

/* nu_t = l_mix^2 |eps(util)|, eq. (mix); l_mix eq. (lmix); y_DES smooth form, eq. (ydes). */
static double eddy_visc(const omesh *M, int c, const ptab *t, const double gt[3][3]) {
  if (!t->enriched) return 0.0;
  double e2 = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double eab = 0.5 * (gt[a][b] + gt[b][a]);
      e2 += eab * eab;
    }
  double eps_norm = sqrt(2.0 * e2);
  double h = M->dye[c] / (M->k + 1);
  double ydes = 0.0;
  if (t->yh > 0.0) ydes = pow(pow(t->yh, -BETA_DES) + pow(C_DES * h, -BETA_DES), -1.0 / BETA_DES);
  double lmix = KAPPA * ydes * (1.0 - exp(-t->yp / APLUS));
  return lmix * lmix * eps_norm;
}

/* Public: evaluate the velocity (ubar+util, 3 values), util, psi, y+ at reference point xi of
 * cell c. out = [u(3), ubar(3), util(3), psi, yplus, nu_t(of u)]. */
void dgo_eval_point(void *h, const double *u, int c, const double *xi, double *out) {
  omesh *M = (omesh *)h;
  ptab t; ptab_alloc(&t, M);
  tabulate(M, c, xi, &t);
  vstate s;
  eval_vel(M, u, c, &t, &s);
  for (int a = 0; a < 3; ++a) { out[a] = s.ub[a] + s.ut[a]; out[3 + a] = s.ub[a]; out[6 + a] = s.ut[a]; }
  out[9] = t.enriched ? t.psi : 0.0;
  out[10] = t.enriched ? t.yp : 0.0;
  out[11] = eddy_visc(M, c, &t, s.gt);
  ptab_free(&t);
}

/* ------------------------------------------------------------------------------------------ */
/* Quadrature bookkeeping                                                                     */
/* ------------------------------------------------------------------------------------------ */

enum { OP_LINEAR = 0, OP_CONVECTIVE = 1, OP_LAPLACE = 2 };

static int inplane_points(const omesh *M, int op) {
  int n = (op == OP_CONVECTIVE) ? (3 * M->k) / 2 + 1 : M->k + 1;
  return n + M->P.extra_q;
}
/* points per reference direction inside cell c */
static void cell_points(const omesh *M, int c, int op, int nq[3]) {
  int n = inplane_points(M, op);
  nq[0] = nq[1] = nq[2] = n;
  if (op != OP_LAPLACE && M->enr[c] >= 0) {
    nq[1] = M->P.q_wall + M->P.extra_q;
    if (M->P.full_q) nq[0] = nq[2] = nq[1];
  }
}

/* Neighbour across face f (d = f/2, side = f%2) of cell c: returns cell or -1 for a wall. */
static int neighbour(const omesh *M, int c, int f) {
  int nx = M->P.nx, ny = M->P.ny, nz = M->P.nz;
  int i = c % nx, j = (c / nx) % ny, kz = c / (nx * ny);
  int d = f / 2, s = f % 2 ? 1 : -1;
  if (d == 0) i = (i + s + nx) % nx;
  else if (d == 2) kz = (kz + s + nz) % nz;
  else { j += s; if (j < 0 || j >= ny) return -1; }
  return cell_id(M, i, j, kz);
}

/* face points per tangential direction: the enriched count in the wall-normal direction if
 * either adjacent cell is enriched (Sec. 4.4) */
static void face_points(const omesh *M, int c, int nb, int d, int op, int *t1, int *t2,
                        int *n_t1, int *n_t2) {
  *t1 = d == 0 ? 1 : 0;
  *t2 = d == 2 ? 1 : 2;
  int n = inplane_points(M, op);
  int enr = op != OP_LAPLACE && (M->enr[c] >= 0 || (nb >= 0 && M->enr[nb] >= 0));
  *n_t1 = ((*t1 == 1 || M->P.full_q) && enr) ? M->P.q_wall + M->P.extra_q : n;
  *n_t2 = ((*t2 == 1 || M->P.full_q) && enr) ? M->P.q_wall + M->P.extra_q : n;
}

/* ------------------------------------------------------------------------------------------ */
/* Operators                                                                                  */
/* ------------------------------------------------------------------------------------------ */

/* y = -L(q,p): SIPG, eq. (ipflux), homogeneous Neumann on walls. */
int dgo_laplace(void *h, const double *p, double *y) {
  omesh *M = (omesh *)h;
  int n3 = M->n1 * M->n1 * M->n1;
  memset(y, 0, sizeof(double) * M->np);
#pragma omp parallel
  {
    ptab t, tn; ptab_alloc(&t, M); ptab_alloc(&tn, M);
    double gx[MAXP], gw[MAXP], gx2[MAXP], gw2[MAXP];
#pragma omp for schedule(dynamic, 4)
    for (int c = 0; c < M->nc; ++c) {
      if (M->active && !M->active[c]) continue;
      double *yc = y + (size_t)c * n3;
      const double *pc = p + (size_t)c * n3;
      int nq[3];
      cell_points(M, c, OP_LAPLACE, nq);
      dgo_gauss(nq[0], gx, gw);
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0) {
            double xi[3] = {gx[q0], gx[q1], gx[q2]};
            tabulate(M, c, xi, &t);
            double dV = fabs(t.detJ) * gw[q0] * gw[q1] * gw[q2];
            double gp[3] = {0, 0, 0};
            for (int i = 0; i < n3; ++i)
              for (int e = 0; e < 3; ++e) gp[e] += t.gphi[3 * i + e] * pc[i];
            for (int i = 0; i < n3; ++i)
              yc[i] += dV * (t.gphi[3 * i] * gp[0] + t.gphi[3 * i + 1] * gp[1] + t.gphi[3 * i + 2] * gp[2]);
          }
      for (int f = 0; f < 6; ++f) {
        int nb = neighbour(M, c, f);
        if (nb < 0) continue;   /* homogeneous Neumann: no wall-face contribution */
        int d = f / 2, side = f % 2, t1, t2, m1, m2;
        face_points(M, c, nb, d, OP_LAPLACE, &t1, &t2, &m1, &m2);
        dgo_gauss(m1, gx, gw); dgo_gauss(m2, gx2, gw2);
        double tau = fmax(M->tau_cell[c], M->tau_cell[nb]);
        const double *pn = p + (size_t)nb * n3;
        for (int b = 0; b < m2; ++b)
          for (int a = 0; a < m1; ++a) {
            double xi[3], xn[3], n[3];
            xi[d] = side; xi[t1] = gx[a]; xi[t2] = gx2[b];
            xn[d] = 1 - side; xn[t1] = gx[a]; xn[t2] = gx2[b];
            tabulate(M, c, xi, &t);
            tabulate(M, nb, xn, &tn);
            double dA = face_geom(t.Ji, t.detJ, d, side, n) * gw[a] * gw2[b];
            double ps = 0, po = 0, gs[3] = {0, 0, 0}, go[3] = {0, 0, 0};
            for (int i = 0; i < n3; ++i) {
              ps += t.phi[i] * pc[i]; po += tn.phi[i] * pn[i];
              for (int e = 0; e < 3; ++e) { gs[e] += t.gphi[3 * i + e] * pc[i]; go[e] += tn.gphi[3 * i + e] * pn[i]; }
            }
            double jump = ps - po;                                      /* [[p]].n_s */
            double flux = 0.5 * ((gs[0] + go[0]) * n[0] + (gs[1] + go[1]) * n[1] + (gs[2] + go[2]) * n[2])
                          - tau * jump;                                 /* P*.n_s */
            for (int i = 0; i < n3; ++i) {
              double dn = t.gphi[3 * i] * n[0] + t.gphi[3 * i + 1] * n[1] + t.gphi[3 * i + 2] * n[2];
              yc[i] -= dA * (0.5 * dn * jump + t.phi[i] * flux);
            }
          }
      }
    }
    ptab_free(&t); ptab_free(&tn);
  }
  return 0;
}

/* Diagonal of the Laplace matrix (own-side terms with the test function as trial function). */
int dgo_laplace_diag(void *h, double *dg) {
  omesh *M = (omesh *)h;
  int n3 = M->n1 * M->n1 * M->n1;
  memset(dg, 0, sizeof(double) * M->np);
#pragma omp parallel
  {
    ptab t, tn; ptab_alloc(&t, M); ptab_alloc(&tn, M);
    double gx[MAXP], gw[MAXP], gx2[MAXP], gw2[MAXP];
#pragma omp for schedule(dynamic, 4)
    for (int c = 0; c < M->nc; ++c) {
      double *dc = dg + (size_t)c * n3;
      int nq[3];
      cell_points(M, c, OP_LAPLACE, nq);
      dgo_gauss(nq[0], gx, gw);
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0) {
            double xi[3] = {gx[q0], gx[q1], gx[q2]};
            tabulate(M, c, xi, &t);
            double dV = fabs(t.detJ) * gw[q0] * gw[q1] * gw[q2];
            for (int i = 0; i < n3; ++i)
              dc[i] += dV * (t.gphi[3 * i] * t.gphi[3 * i] + t.gphi[3 * i + 1] * t.gphi[3 * i + 1] +
                             t.gphi[3 * i + 2] * t.gphi[3 * i + 2]);
          }
      for (int f = 0; f < 6; ++f) {
        int nb = neighbour(M, c, f);
        if (nb < 0) continue;
        int d = f / 2, side = f % 2, t1, t2, m1, m2;
        face_points(M, c, nb, d, OP_LAPLACE, &t1, &t2, &m1, &m2);
        dgo_gauss(m1, gx, gw); dgo_gauss(m2, gx2, gw2);
        double tau = fmax(M->tau_cell[c], M->tau_cell[nb]);
        for (int b = 0; b < m2; ++b)
          for (int a = 0; a < m1; ++a) {
            double xi[3], n[3];
            xi[d] = side; xi[t1] = gx[a]; xi[t2] = gx2[b];
            tabulate(M, c, xi, &t);
            double dA = face_geom(t.Ji, t.detJ, d, side, n) * gw[a] * gw2[b];
            if (nb == c) {   /* one cell across a periodic direction: trial also on the far side */
              double xn[3];
              xn[d] = 1 - side; xn[t1] = gx[a]; xn[t2] = gx2[b];
              tabulate(M, c, xn, &tn);
            }
            for (int i = 0; i < n3; ++i) {
              double dn = t.gphi[3 * i] * n[0] + t.gphi[3 * i + 1] * n[1] + t.gphi[3 * i + 2] * n[2];
              double po = 0.0, dno = 0.0;
              if (nb == c) {
                po = tn.phi[i];
                dno = tn.gphi[3 * i] * n[0] + tn.gphi[3 * i + 1] * n[1] + tn.gphi[3 * i + 2] * n[2];
              }
              double jump = t.phi[i] - po;
              dc[i] -= dA * (0.5 * dn * jump + t.phi[i] * (0.5 * (dn + dno) - tau * jump));
            }
          }
      }
    }
    ptab_free(&t); ptab_free(&tn);
  }
  return 0;
}

/* b = -C(q,u) = (grad q, u) - (q, {{u}}.n); {{u}} = u^- on walls; u = ubar + util. */
int dgo_divergence(void *h, const double *u, double *b) {
  omesh *M = (omesh *)h;
  int n3 = M->n1 * M->n1 * M->n1;
  memset(b, 0, sizeof(double) * M->np);
#pragma omp parallel
  {
    ptab t, tn; ptab_alloc(&t, M); ptab_alloc(&tn, M);
    double gx[MAXP], gw[MAXP], gy[MAXP], gwy[MAXP], gx2[MAXP], gw2[MAXP];
#pragma omp for schedule(dynamic, 4)
    for (int c = 0; c < M->nc; ++c) {
      if (M->active && !M->active[c]) continue;
      double *bc = b + (size_t)c * n3;
      int nq[3];
      cell_points(M, c, OP_LINEAR, nq);
      dgo_gauss(nq[0], gx, gw); dgo_gauss(nq[1], gy, gwy);
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0) {
            double xi[3] = {gx[q0], gy[q1], gx[q2]};
            tabulate(M, c, xi, &t);
            double dV = fabs(t.detJ) * gw[q0] * gwy[q1] * gw[q2];
            vstate s; eval_vel(M, u, c, &t, &s);
            double uu[3] = {s.ub[0] + s.ut[0], s.ub[1] + s.ut[1], s.ub[2] + s.ut[2]};
            for (int i = 0; i < n3; ++i)
              bc[i] += dV * (t.gphi[3 * i] * uu[0] + t.gphi[3 * i + 1] * uu[1] + t.gphi[3 * i + 2] * uu[2]);
          }
      for (int f = 0; f < 6; ++f) {
        int nb = neighbour(M, c, f);
        int d = f / 2, side = f % 2, t1, t2, m1, m2;
        face_points(M, c, nb, d, OP_LINEAR, &t1, &t2, &m1, &m2);
        dgo_gauss(m1, gx, gw); dgo_gauss(m2, gx2, gw2);
        for (int bq = 0; bq < m2; ++bq)
          for (int a = 0; a < m1; ++a) {
            double xi[3], xn[3], n[3];
            xi[d] = side; xi[t1] = gx[a]; xi[t2] = gx2[bq];
            tabulate(M, c, xi, &t);
            double dA = face_geom(t.Ji, t.detJ, d, side, n) * gw[a] * gw2[bq];
            vstate s, so; eval_vel(M, u, c, &t, &s);
            double avg[3];
            if (nb >= 0) {
              xn[d] = 1 - side; xn[t1] = gx[a]; xn[t2] = gx2[bq];
              tabulate(M, nb, xn, &tn);
              eval_vel(M, u, nb, &tn, &so);
              for (int e = 0; e < 3; ++e) avg[e] = 0.5 * (s.ub[e] + s.ut[e] + so.ub[e] + so.ut[e]);
            } else {
              for (int e = 0; e < 3; ++e) avg[e] = s.ub[e] + s.ut[e];   /* wall: interior value */
            }
            double fn = avg[0] * n[0] + avg[1] * n[1] + avg[2] * n[2];
            for (int i = 0; i < n3; ++i) bc[i] -= dA * t.phi[i] * fn;
          }
      }
    }
    ptab_free(&t); ptab_free(&tn);
  }
  return 0;
}

/* Output index helpers for velocity-space vectors. */
static inline double *std_out(const omesh *M, double *y, int c, int a) {
  return y + ((size_t)c * 3 + a) * M->n1 * M->n1 * M->n1;
}
static inline double *enr_out(const omesh *M, double *y, int c, int a) {
  return y + 3L * M->np + ((size_t)M->enr[c] * 3 + a) * M->nef;
}

/* y = F^c(v,u) = -(grad v, u x u) + (v, F^c*.n), local Lax-Friedrichs flux; walls: u+ = -u-. */
int dgo_convective(void *h, const double *u, double *y) {
  omesh *M = (omesh *)h;
  int n3 = M->n1 * M->n1 * M->n1;
  memset(y, 0, sizeof(double) * M->nu);
#pragma omp parallel
  {
    ptab t, tn; ptab_alloc(&t, M); ptab_alloc(&tn, M);
    double gx[MAXP], gw[MAXP], gy[MAXP], gwy[MAXP], gx2[MAXP], gw2[MAXP];
#pragma omp for schedule(dynamic, 4)
    for (int c = 0; c < M->nc; ++c) {
      if (M->active && !M->active[c]) continue;
      int enriched = M->enr[c] >= 0;
      int nq[3];
      cell_points(M, c, OP_CONVECTIVE, nq);
      dgo_gauss(nq[0], gx, gw); dgo_gauss(nq[1], gy, gwy);
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0) {
            double xi[3] = {gx[q0], gy[q1], gx[q2]};
            tabulate(M, c, xi, &t);
            double dV = fabs(t.detJ) * gw[q0] * gwy[q1] * gw[q2];
            vstate s; eval_vel(M, u, c, &t, &s);
            double uu[3] = {s.ub[0] + s.ut[0], s.ub[1] + s.ut[1], s.ub[2] + s.ut[2]};
            for (int a = 0; a < 3; ++a) {
              double *ya = std_out(M, y, c, a);
              for (int i = 0; i < n3; ++i) {
                double ug = t.gphi[3 * i] * uu[0] + t.gphi[3 * i + 1] * uu[1] + t.gphi[3 * i + 2] * uu[2];
                ya[i] -= dV * uu[a] * ug;
              }
              if (enriched) {
                double *ye = enr_out(M, y, c, a);
                for (int v = 0; v < M->nef; ++v) {
                  double ug = t.egphi[v][0] * uu[0] + t.egphi[v][1] * uu[1] + t.egphi[v][2] * uu[2];
                  ye[v] -= dV * uu[a] * ug;
                }
              }
            }
          }
      for (int f = 0; f < 6; ++f) {
        int nb = neighbour(M, c, f);
        int d = f / 2, side = f % 2, t1, t2, m1, m2;
        face_points(M, c, nb, d, OP_CONVECTIVE, &t1, &t2, &m1, &m2);
        dgo_gauss(m1, gx, gw); dgo_gauss(m2, gx2, gw2);
        for (int bq = 0; bq < m2; ++bq)
          for (int a = 0; a < m1; ++a) {
            double xi[3], xn[3], n[3];
            xi[d] = side; xi[t1] = gx[a]; xi[t2] = gx2[bq];
            tabulate(M, c, xi, &t);
            double dA = face_geom(t.Ji, t.detJ, d, side, n) * gw[a] * gw2[bq];
            vstate s, so; eval_vel(M, u, c, &t, &s);
            double um[3], up[3];
            for (int e = 0; e < 3; ++e) um[e] = s.ub[e] + s.ut[e];
            if (nb >= 0) {
              xn[d] = 1 - side; xn[t1] = gx[a]; xn[t2] = gx2[bq];
              tabulate(M, nb, xn, &tn);
              eval_vel(M, u, nb, &tn, &so);
              for (int e = 0; e < 3; ++e) up[e] = so.ub[e] + so.ut[e];
            } else {
              for (int e = 0; e < 3; ++e) up[e] = -um[e];   /* mirror principle, g = 0 */
            }
            double unm = um[0] * n[0] + um[1] * n[1] + um[2] * n[2];
            double unp = up[0] * n[0] + up[1] * n[1] + up[2] * n[2];
            double lam = fmax(2.0 * fabs(unm), 2.0 * fabs(unp));
            double F[3];
            for (int e = 0; e < 3; ++e)
              F[e] = 0.5 * (um[e] * unm + up[e] * unp) + 0.5 * lam * (um[e] - up[e]);
            for (int e = 0; e < 3; ++e) {
              double *ya = std_out(M, y, c, e);
              for (int i = 0; i < n3; ++i) ya[i] += dA * t.phi[i] * F[e];
              if (enriched) {
                double *ye = enr_out(M, y, c, e);
                for (int v = 0; v < M->nef; ++v) ye[v] += dA * t.ephi[v] * F[e];
              }
            }
          }
      }
    }
    ptab_free(&t); ptab_free(&tn);
  }
  return 0;
}

/* Contract grad(test) of a vector test function e_a * g with a tensor T: sum_b g_b T[a][b]. */
static inline double gdot(const double *g, const double T[3][3], int a) {
  return g[0] * T[a][0] + g[1] * T[a][1] + g[2] * T[a][2];
}
/* eps(test):T for symmetric T equals grad(test):T. 2*eps(w) from a gradient. */
static inline void two_eps(const double G[3][3], double f, double T[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) T[a][b] = f * (G[a][b] + G[b][a]);
}

/* y = -F^nu(vbar, vtil; ubar, util), eq. (viscous_multiscale), with nu_t evaluated from u_frz
 * at every quadrature point and frozen; harmonic weights eq. (harmweights); clipped viscosity
 * eq. (minvt) in the (vbar, util) volume term; mirror state on walls; penalty uses nu only. */
int dgo_viscous(void *h, const double *u_frz, const double *u, double *y) {
  omesh *M = (omesh *)h;
  int n3 = M->n1 * M->n1 * M->n1;
  const double nu = M->P.nu;
  memset(y, 0, sizeof(double) * M->nu);
#pragma omp parallel
  {
    ptab t, tn; ptab_alloc(&t, M); ptab_alloc(&tn, M);
    double gx[MAXP], gw[MAXP], gy[MAXP], gwy[MAXP], gx2[MAXP], gw2[MAXP];
#pragma omp for schedule(dynamic, 4)
    for (int c = 0; c < M->nc; ++c) {
      if (M->active && !M->active[c]) continue;
      int enr_c = M->enr[c] >= 0;
      int nq[3];
      cell_points(M, c, OP_LINEAR, nq);
      dgo_gauss(nq[0], gx, gw); dgo_gauss(nq[1], gy, gwy);
      /* volume terms */
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0) {
            double xi[3] = {gx[q0], gy[q1], gx[q2]};
            tabulate(M, c, xi, &t);
            double dV = fabs(t.detJ) * gw[q0] * gwy[q1] * gw[q2];
            vstate s, sf; eval_vel(M, u, c, &t, &s);
            double Tb[3][3], Tth[3][3], Ttf[3][3];
            two_eps(s.gb, nu, Tb);                    /* F^nu(ubar) */
            if (enr_c) {
              eval_vel(M, u_frz, c, &t, &sf);
              double nut = eddy_visc(M, c, &t, sf.gt);
              double nuh = fmin(nu + nut, 2.0 * sqrt(nu * (nu + nut)));   /* eq. (minvt) */
              two_eps(s.gt, nuh, Tth);
              two_eps(s.gt, nu + nut, Ttf);
              for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) Tb[a][b] += Tth[a][b];
            }
            for (int a = 0; a < 3; ++a) {
              double *ya = std_out(M, y, c, a);
              for (int i = 0; i < n3; ++i) ya[i] += dV * gdot(t.gphi + 3 * i, Tb, a);
              if (enr_c) {
                double *ye = enr_out(M, y, c, a);
                for (int v = 0; v < M->nef; ++v) ye[v] += dV * gdot(t.egphi[v], Ttf, a);
              }
            }
          }
      /* face terms, from the side of cell c */
      for (int f = 0; f < 6; ++f) {
        int nb = neighbour(M, c, f);
        int d = f / 2, side = f % 2, t1, t2, m1, m2;
        face_points(M, c, nb, d, OP_LINEAR, &t1, &t2, &m1, &m2);
        dgo_gauss(m1, gx, gw); dgo_gauss(m2, gx2, gw2);
        int enr_o = nb >= 0 ? M->enr[nb] >= 0 : enr_c;   /* mirror side carries c's class */
        int both = enr_c && enr_o;                        /* d Omega~_e (incl. enriched walls) */
        int iface = enr_c != enr_o;                       /* d Omega~^I_e */
        double tau = nb >= 0 ? fmax(M->tau_cell[c], M->tau_cell[nb]) : WALL_PENALTY * M->tau_cell[c];
        for (int bq = 0; bq < m2; ++bq)
          for (int a = 0; a < m1; ++a) {
            double xi[3], xn[3], n[3];
            xi[d] = side; xi[t1] = gx[a]; xi[t2] = gx2[bq];
            tabulate(M, c, xi, &t);
            double dA = face_geom(t.Ji, t.detJ, d, side, n) * gw[a] * gw2[bq];
            vstate s, so, sf, sfo;
            eval_vel(M, u, c, &t, &s);
            double nut_s = 0.0, nut_o = 0.0;
            if (enr_c) { eval_vel(M, u_frz, c, &t, &sf); nut_s = eddy_visc(M, c, &t, sf.gt); }
            if (nb >= 0) {
              xn[d] = 1 - side; xn[t1] = gx[a]; xn[t2] = gx2[bq];
              tabulate(M, nb, xn, &tn);
              eval_vel(M, u, nb, &tn, &so);
              if (enr_o) { eval_vel(M, u_frz, nb, &tn, &sfo); nut_o = eddy_visc(M, nb, &tn, sfo.gt); }
            } else {
              /* mirror principle: u+ = -u-, grad u+ = grad u-, nu_t+ = nu_t- */
              so = s;
              for (int e = 0; e < 3; ++e) { so.ub[e] = -s.ub[e]; so.ut[e] = -s.ut[e]; }
              nut_o = nut_s;
            }
            /* jumps [[w]] = (w_s - w_o) x n (n outward of c) */
            double jb[3], jt[3], jtot[3];
            for (int e = 0; e < 3; ++e) {
              jb[e] = s.ub[e] - so.ub[e];
              jt[e] = s.ut[e] - so.ut[e];
              jtot[e] = jb[e] + jt[e];
            }
            /* standard averages: {{F^nu(ubar)}}.n */
            double Fbs[3][3], Fbo[3][3], avgb_n[3];
            two_eps(s.gb, nu, Fbs); two_eps(so.gb, nu, Fbo);
            for (int e = 0; e < 3; ++e)
              avgb_n[e] = 0.5 * ((Fbs[e][0] + Fbo[e][0]) * n[0] + (Fbs[e][1] + Fbo[e][1]) * n[1] +
                                 (Fbs[e][2] + Fbo[e][2]) * n[2]);
            /* weighted enriched average {{F^{nu+nut}(util)}}_w.n on d Omega~_e */
            double wt_s = 0.5, avgt_n[3] = {0, 0, 0};
            if (both) {
              double den = 2.0 * nu + nut_s + nut_o;
              wt_s = (nu + nut_o) / den;
              double wt_o = (nu + nut_s) / den;
              double Fts[3][3], Fto[3][3];
              two_eps(s.gt, nu + nut_s, Fts); two_eps(so.gt, nu + nut_o, Fto);
              for (int e = 0; e < 3; ++e)
                avgt_n[e] = (wt_s * Fts[e][0] + wt_o * Fto[e][0]) * n[0] +
                            (wt_s * Fts[e][1] + wt_o * Fto[e][1]) * n[1] +
                            (wt_s * Fts[e][2] + wt_o * Fto[e][2]) * n[2];
            }
            /* standard test functions vbar = phi_i e_a */
            for (int ea = 0; ea < 3; ++ea) {
              double *ya = std_out(M, y, c, ea);
              /* value coefficient */
              double cv = -avgb_n[ea] + tau * nu * jtot[ea];
              if (both) cv -= avgt_n[ea];
              /* gradient coefficient: (1/2 F^nu(vbar)) : [[ubar]] (+ [[util]] on the interface)
               * = nu * (grad v + grad v^T)/2... written as g . w with w_b = contraction */
              double jadj[3];
              for (int e = 0; e < 3; ++e) jadj[e] = jb[e] + (iface ? jt[e] : 0.0);
              for (int i = 0; i < n3; ++i) {
                const double *g = t.gphi + 3 * i;
                /* (1/2 F^nu(phi e_a)) : (j x n) = nu eps(e_a x g) : (j x n)
                 *                             = nu/2 (j_a (g.n) + n_a (g.j)) */
                double gn = g[0] * n[0] + g[1] * n[1] + g[2] * n[2];
                double gj = g[0] * jadj[0] + g[1] * jadj[1] + g[2] * jadj[2];
                double adj = nu * 0.5 * (jadj[ea] * gn + n[ea] * gj);
                ya[i] += dA * (adj + t.phi[i] * cv);
              }
            }
            /* enriched test functions vtil = psi N_B e_a */
            if (enr_c) {
              for (int ea = 0; ea < 3; ++ea) {
                double *ye = enr_out(M, y, c, ea);
                double cv = tau * nu * jtot[ea];
                if (both) cv -= avgt_n[ea];
                if (iface) cv -= avgb_n[ea];
                for (int v = 0; v < M->nef; ++v) {
                  double adj = 0.0;
                  if (both) {
                    /* (w F^{nu+nut}(vtil), [[util]] + [[ubar]]) */
                    const double *g = t.egphi[v];
                    double gn = g[0] * n[0] + g[1] * n[1] + g[2] * n[2];
                    double gj = g[0] * jtot[0] + g[1] * jtot[1] + g[2] * jtot[2];
                    adj = wt_s * (nu + nut_s) * (jtot[ea] * gn + n[ea] * gj);
                  }
                  ye[v] += dA * (adj + t.ephi[v] * cv);
                }
              }
            }
          }
      }
    }
    ptab_free(&t); ptab_free(&tn);
  }
  return 0;
}

/* nu_t at every volume quadrature point of enriched cell e (points ordered x fastest, then y
 * (q_wall points), then z), evaluated from u. Used by tests to check clipping statistics. */
int dgo_nut_cell(void *h, const double *u, int e, double *out) {
  omesh *M = (omesh *)h;
  if (e < 0 || e >= M->ne) return -1;
  int c = M->enr_cell[e], nq[3];
  cell_points(M, c, OP_LINEAR, nq);
  double gx[MAXP], gw[MAXP], gy[MAXP], gwy[MAXP];
  dgo_gauss(nq[0], gx, gw); dgo_gauss(nq[1], gy, gwy);
  ptab t; ptab_alloc(&t, M);
  int idx = 0;
  for (int q2 = 0; q2 < nq[2]; ++q2)
    for (int q1 = 0; q1 < nq[1]; ++q1)
      for (int q0 = 0; q0 < nq[0]; ++q0) {
        double xi[3] = {gx[q0], gy[q1], gx[q2]};
        tabulate(M, c, xi, &t);
        vstate s; eval_vel(M, u, c, &t, &s);
        out[idx++] = eddy_visc(M, c, &t, s.gt);
      }
  ptab_free(&t);
  return idx;
}

/* Sum of |detJ| w over all cells (domain volume). */
double dgo_volume(void *h) {
  omesh *M = (omesh *)h;
  int n = M->n1 + 2;
  double gx[MAXP], gw[MAXP], V = 0.0;
  dgo_gauss(n, gx, gw);
  for (int c = 0; c < M->nc; ++c)
    for (int q2 = 0; q2 < n; ++q2)
      for (int q1 = 0; q1 < n; ++q1)
        for (int q0 = 0; q0 < n; ++q0) {
          double xi[3] = {gx[q0], gx[q1], gx[q2]}, J[3][3], Ji[3][3], det;
          map_point(M, c, xi, NULL, J, &det, Ji);
          V += fabs(det) * gw[q0] * gw[q1] * gw[q2];
        }
  return V;
}

/* ------------------------------------------------------------------------------------------ */
/* Solver: CG on -L p = b restricted to zero-mean vectors (null space = constants)            */
/* ------------------------------------------------------------------------------------------ */

static double dot(const double *a, const double *b, long n) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s)
  for (long i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static void remove_mean(double *v, long n) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += v[i];
  s /= (double)n;
  for (long i = 0; i < n; ++i) v[i] -= s;
}

/* Jacobi-preconditioned CG. b is projected to 1^T b = 0; p returned with 1^T p = 0.
 * Stops when ||b - A p||_2 / ||b||_2 <= rtol (true residual re-checked at the end). */
int dgo_solve_cg(void *h, const double *b_in, double *p, double rtol, int maxit, int *iters,
                 double *relres) {
  omesh *M = (omesh *)h;
  long n = M->np;
  double *b = malloc(sizeof(double) * n), *r = malloc(sizeof(double) * n),
         *z = malloc(sizeof(double) * n), *d = malloc(sizeof(double) * n),
         *q = malloc(sizeof(double) * n), *dg = malloc(sizeof(double) * n);
  memcpy(b, b_in, sizeof(double) * n);
  remove_mean(b, n);
  dgo_laplace_diag(h, dg);
  double bn = sqrt(dot(b, b, n));
  memset(p, 0, sizeof(double) * n);
  memcpy(r, b, sizeof(double) * n);
  int it = 0;
  double res = bn > 0 ? 1.0 : 0.0;
  if (bn == 0.0) { *iters = 0; *relres = 0.0; goto done; }
  for (long i = 0; i < n; ++i) z[i] = r[i] / dg[i];
  remove_mean(z, n);
  memcpy(d, z, sizeof(double) * n);
  double rz = dot(r, z, n);
  for (it = 1; it <= maxit; ++it) {
    dgo_laplace(h, d, q);
    double alpha = rz / dot(d, q, n);
    for (long i = 0; i < n; ++i) { p[i] += alpha * d[i]; r[i] -= alpha * q[i]; }
    res = sqrt(dot(r, r, n)) / bn;
    if (res <= rtol) break;
    for (long i = 0; i < n; ++i) z[i] = r[i] / dg[i];
    remove_mean(z, n);
    double rz2 = dot(r, z, n);
    double beta = rz2 / rz;
    rz = rz2;
    for (long i = 0; i < n; ++i) d[i] = z[i] + beta * d[i];
  }
  remove_mean(p, n);
  dgo_laplace(h, p, q);
  for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
  *relres = sqrt(dot(r, r, n)) / bn;
  *iters = it > maxit ? maxit : it;
done:
  free(b); free(r); free(z); free(d); free(q); free(dg);
  return 0;
}

int dgo_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void dgo_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* y = M_e(v, u) = (v, u) over every cell (Sec. 4.2 mass term) for the velocity space: standard test
 * functions and, in enriched cells, the enriched ones psi N_B e_a; u = ubar + util; linear-term points
 * (q_wall wall-normal points in enriched cells). No face terms. */
int dgo_vmass(void *h, const double *u, double *y) {
  omesh *M = (omesh *)h;
  int n3 = M->n1 * M->n1 * M->n1;
  memset(y, 0, sizeof(double) * M->nu);
#pragma omp parallel
  {
    ptab t; ptab_alloc(&t, M);
    double gx[MAXP], gw[MAXP], gy[MAXP], gwy[MAXP];
#pragma omp for schedule(dynamic, 4)
    for (int c = 0; c < M->nc; ++c) {
      if (M->active && !M->active[c]) continue;
      int nq[3];
      cell_points(M, c, OP_LINEAR, nq);
      dgo_gauss(nq[0], gx, gw); dgo_gauss(nq[1], gy, gwy);
      int en = M->enr[c];
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0) {
            double xi[3] = {gx[q0], gy[q1], gx[q2]};
            tabulate(M, c, xi, &t);
            double dV = fabs(t.detJ) * gw[q0] * gwy[q1] * gw[q2];
            vstate s; eval_vel(M, u, c, &t, &s);
            for (int a = 0; a < 3; ++a) {
              double va = dV * (s.ub[a] + s.ut[a]);
              double *yc = y + ((size_t)c * 3 + a) * n3;
              for (int i = 0; i < n3; ++i) yc[i] += t.phi[i] * va;
              if (en >= 0) {
                double *ye = y + 3L * M->np + ((size_t)en * 3 + a) * M->nef;
                for (int v = 0; v < M->nef; ++v) ye[v] += t.ephi[v] * va;
              }
            }
          }
    }
    ptab_free(&t);
  }
  return 0;
}

/* y = M p, the pressure-space mass matrix (Sec. 4.2 mass term, scalar), k+1 Gauss points. */
int dgo_mass(void *h, const double *p, double *y) {
  omesh *M = (omesh *)h;
  int n3 = M->n1 * M->n1 * M->n1;
  memset(y, 0, sizeof(double) * M->np);
#pragma omp parallel
  {
    ptab t; ptab_alloc(&t, M);
    double gx[MAXP], gw[MAXP];
#pragma omp for schedule(dynamic, 4)
    for (int c = 0; c < M->nc; ++c) {
      int nq[3];
      cell_points(M, c, OP_LAPLACE, nq);
      dgo_gauss(nq[0], gx, gw);
      const double *pc = p + (size_t)c * n3;
      double *yc = y + (size_t)c * n3;
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0) {
            double xi[3] = {gx[q0], gx[q1], gx[q2]};
            tabulate(M, c, xi, &t);
            double dV = fabs(t.detJ) * gw[q0] * gw[q1] * gw[q2], v = 0.0;
            for (int i = 0; i < n3; ++i) v += t.phi[i] * pc[i];
            for (int i = 0; i < n3; ++i) yc[i] += dV * t.phi[i] * v;
          }
    }
    ptab_free(&t);
  }
  return 0;
}


/* ----------------------------------------------------------------------------------------------
 * Wall shear stress on the linear wall nodes (Sec. 3.2): for wall node B,
 *   tau_w,B = || int_wall N_B tau_w dA || / int_wall N_B dA,   tau_w = rho nu (grad u_h) . n,
 * the numerator integrated per component before the norm. N_B are the continuous bilinear
 * functions of the wall vertices (periodic in x and z), u_h = ubar + utilde with the current
 * enrichment, k+1 Gauss points per tangential direction on each wall face, rho = 1.
 * Wall nodes: index wall * nx * nz + i + nx * k (wall 0 bottom, 1 top).
 * Off-wall vertices of enriched cells carry the value of the wall node that defines their y_B.
 * ---------------------------------------------------------------------------------------------- */
int dgo_wall_nodes(void *h) {
  omesh *M = (omesh *)h;
  return 2 * M->P.nx * M->P.nz;
}

/* Switch-off of the wall model (Sec. 3.2): a wall-nearest enriched cell is switched off when every
 * point of its velocity point set (k+1 in-plane, q_w wall-normal) has y+ < yp_off, with y+ from the
 * linear y_h and tau_w,h of its vertices; enriched cells further from the wall follow the
 * wall-nearest cell of their column. A switched-off cell is a standard cell for every operator
 * (point sets and face classes included); its enrichment coefficients are kept at zero. */
static void apply_switch(omesh *M) {
  const int nx = M->P.nx, ny = M->P.ny, L = M->P.n_layers, n1 = M->n1, qw = M->P.q_wall + M->P.extra_q;
  double gx[MAXP], gw[MAXP], gy[MAXP], gwy[MAXP];
  dgo_gauss(n1 + M->P.extra_q, gx, gw);
  dgo_gauss(qw, gy, gwy);
  const int nin = M->P.full_q ? qw : n1 + M->P.extra_q;
  if (M->P.full_q) dgo_gauss(qw, gx, gw);
  for (int c = 0; c < M->nc; ++c) {
    int e = M->slot[c];
    if (e < 0) continue;
    int i = c % nx, j = (c / nx) % ny, kz = c / (nx * ny);
    int jw = (j < L) ? 0 : ny - 1;                 /* wall-nearest row of this column */
    int ew = M->slot[cell_id(M, i, jw, kz)];
    double ymax = 0.0;
    for (int q2 = 0; q2 < nin; ++q2)
      for (int q1 = 0; q1 < qw; ++q1)
        for (int q0 = 0; q0 < nin; ++q0) {
          double xi[3] = {gx[q0], gy[q1], gx[q2]}, N8[8], g8[8][3], yh = 0.0, th = 0.0;
          q1_basis(8, xi, N8, g8);
          for (int v = 0; v < 8; ++v) { yh += N8[v] * M->ywall[8 * ew + v]; th += N8[v] * M->tauv[8 * ew + v]; }
          double yp = yh * sqrt(th) / M->P.nu;
          if (yp > ymax) ymax = yp;
        }
    M->enr[c] = ymax < M->yp_off ? -1 : e;
  }
}

void dgo_set_tau_nodes(void *h, const double *tn) {
  omesh *M = (omesh *)h;
  for (int i = 0; i < 8 * M->ne; ++i) M->tauv[i] = tn[M->tsrc[i]];
  apply_switch(M);
}

void dgo_set_switch(void *h, double yp_off) {
  omesh *M = (omesh *)h;
  M->yp_off = yp_off;
  apply_switch(M);
}

int dgo_active(void *h, int *on) {
  omesh *M = (omesh *)h;
  int n = 0;
  for (int e = 0; e < M->ne; ++e) {
    on[e] = M->enr[M->enr_cell[e]] >= 0;
    n += on[e];
  }
  return n;
}

int dgo_wall_shear(void *h, const double *u, double *tn) {
  omesh *M = (omesh *)h;
  const int nx = M->P.nx, ny = M->P.ny, nz = M->P.nz, nn = 2 * nx * nz, n1 = M->n1;
  double *num = (double *)calloc((size_t)3 * nn, sizeof(double));
  double *den = (double *)calloc((size_t)nn, sizeof(double));
  double gx[MAXP], gw[MAXP];
  ptab t; ptab_alloc(&t, M);
  for (int wall = 0; wall < 2; ++wall)
    for (int kz = 0; kz < nz; ++kz)
      for (int i = 0; i < nx; ++i) {
        const int j = wall ? ny - 1 : 0, c = cell_id(M, i, j, kz);
        /* k+1 points per direction; q_w on the wall faces of enriched cells under the q_w^3 rule */
        const int nf = (M->P.full_q && M->enr[c] >= 0) ? M->P.q_wall : n1;
        dgo_gauss(nf, gx, gw);
        for (int q2 = 0; q2 < nf; ++q2)
          for (int q0 = 0; q0 < nf; ++q0) {
            double xi[3] = {gx[q0], wall ? 1.0 : 0.0, gx[q2]}, nrm[3];
            tabulate(M, c, xi, &t);
            double dA = face_geom(t.Ji, t.detJ, 1, wall, nrm) * gw[q0] * gw[q2];
            vstate st; eval_vel(M, u, c, &t, &st);
            double tw[3];
            for (int a = 0; a < 3; ++a) {
              tw[a] = 0.0;
              for (int d = 0; d < 3; ++d) tw[a] += M->P.nu * (st.gb[a][d] + st.gt[a][d]) * nrm[d];
            }
            /* the four wall vertices of the face and their bilinear functions */
            for (int b = 0; b < 4; ++b) {
              int bi = b & 1, bk = b >> 1;
              double Nb = (bi ? xi[0] : 1.0 - xi[0]) * (bk ? xi[2] : 1.0 - xi[2]);
              int node = wall * nx * nz + (i + bi) % nx + nx * ((kz + bk) % nz);
              for (int a = 0; a < 3; ++a) num[3 * node + a] += Nb * tw[a] * dA;
              den[node] += Nb * dA;
            }
          }
      }
  ptab_free(&t);
  for (int b = 0; b < nn; ++b)
    tn[b] = sqrt(num[3 * b] * num[3 * b] + num[3 * b + 1] * num[3 * b + 1] + num[3 * b + 2] * num[3 * b + 2]) / den[b];
  free(num); free(den);
  return nn;
}

/* ----------------------------------------------------------------------------------------------
 * Cell-wise L2 projection onto the space of a new nodal wall shear stress (Sec. 3.2, eq. l2):
 * in every enriched cell, u_new in V_new with int v . u_new = int v . u_old for all v in V_new
 * (per component; V_new = standard Q_k plus psi_new N^l), integrated with the cell's velocity
 * point set (k+1 points in-plane, q_w wall-normal). The other cells' spaces do not change and
 * their coefficients are copied. The cell system is solved by Gaussian elimination with partial
 * pivoting. The mesh keeps tau_new afterwards.
 * ---------------------------------------------------------------------------------------------- */
static int solve_dense(int N, double *A, double *B, int nrhs) {
  /* A: N x N row-major, B: N x nrhs row-major; overwritten with the solution */
  for (int k = 0; k < N; ++k) {
    int piv = k;
    for (int i = k + 1; i < N; ++i)
      if (fabs(A[(size_t)i * N + k]) > fabs(A[(size_t)piv * N + k])) piv = i;
    if (A[(size_t)piv * N + k] == 0.0) return -1;
    if (piv != k) {
      for (int j = 0; j < N; ++j) {
        double t = A[(size_t)k * N + j]; A[(size_t)k * N + j] = A[(size_t)piv * N + j]; A[(size_t)piv * N + j] = t;
      }
      for (int r = 0; r < nrhs; ++r) {
        double t = B[(size_t)k * nrhs + r]; B[(size_t)k * nrhs + r] = B[(size_t)piv * nrhs + r]; B[(size_t)piv * nrhs + r] = t;
      }
    }
    for (int i = k + 1; i < N; ++i) {
      double f = A[(size_t)i * N + k] / A[(size_t)k * N + k];
      if (f == 0.0) continue;
      for (int j = k; j < N; ++j) A[(size_t)i * N + j] -= f * A[(size_t)k * N + j];
      for (int r = 0; r < nrhs; ++r) B[(size_t)i * nrhs + r] -= f * B[(size_t)k * nrhs + r];
    }
  }
  for (int k = N - 1; k >= 0; --k)
    for (int r = 0; r < nrhs; ++r) {
      double s = B[(size_t)k * nrhs + r];
      for (int j = k + 1; j < N; ++j) s -= A[(size_t)k * N + j] * B[(size_t)j * nrhs + r];
      B[(size_t)k * nrhs + r] = s / A[(size_t)k * N + k];
    }
  return 0;
}

int dgo_project(void *h, const double *tau_new, const double *u_old, double *u_new) {
  omesh *M = (omesh *)h;
  const int n3 = M->n1 * M->n1 * M->n1, nef = M->nef, N = n3 + nef;
  memcpy(u_new, u_old, sizeof(double) * M->nu);
  if (M->ne == 0) { dgo_set_tau_nodes(h, tau_new); return 0; }
  /* old field at the points of every enriched cell */
  /* the wall cells' velocity point set, whether switched on or off */
  const int qin = M->P.full_q ? M->P.q_wall + M->P.extra_q : M->n1 + M->P.extra_q;
  const int nq[3] = {qin, M->P.q_wall + M->P.extra_q, qin};
  const int npts = nq[0] * nq[1] * nq[2];
  double gx[MAXP], gw[MAXP], gy[MAXP], gwy[MAXP];
  dgo_gauss(nq[0], gx, gw); dgo_gauss(nq[1], gy, gwy);
  double *uold = (double *)malloc(sizeof(double) * (size_t)M->ne * npts * 3);
  int status = 0;
#pragma omp parallel
  {
    ptab t; ptab_alloc(&t, M);
#pragma omp for schedule(dynamic, 1)
    for (int e = 0; e < M->ne; ++e) {
      int c = M->enr_cell[e], q = 0;
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0, ++q) {
            double xi[3] = {gx[q0], gy[q1], gx[q2]};
            tabulate(M, c, xi, &t);
            vstate s; eval_vel(M, u_old, c, &t, &s);
            for (int a = 0; a < 3; ++a) uold[((size_t)e * npts + q) * 3 + a] = s.ub[a] + s.ut[a];
          }
    }
    ptab_free(&t);
  }
  dgo_set_tau_nodes(h, tau_new);
#pragma omp parallel
  {
    ptab t; ptab_alloc(&t, M);
    double *A = (double *)malloc(sizeof(double) * (size_t)N * N);
    double *B = (double *)malloc(sizeof(double) * (size_t)N * 3);
    double *phi = (double *)malloc(sizeof(double) * N);
#pragma omp for schedule(dynamic, 1)
    for (int e = 0; e < M->ne; ++e) {
      int c = M->enr_cell[e], q = 0;
      const int Nc = M->enr[c] >= 0 ? N : n3;   /* switched off: standard functions only */
      memset(A, 0, sizeof(double) * (size_t)N * N);
      memset(B, 0, sizeof(double) * (size_t)N * 3);
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0, ++q) {
            double xi[3] = {gx[q0], gy[q1], gx[q2]};
            tabulate(M, c, xi, &t);
            double dV = fabs(t.detJ) * gw[q0] * gwy[q1] * gw[q2];
            for (int i = 0; i < n3; ++i) phi[i] = t.phi[i];
            for (int v = 0; v < nef; ++v) phi[n3 + v] = t.enriched ? t.ephi[v] : 0.0;
            for (int i = 0; i < Nc; ++i) {
              double wi = dV * phi[i];
              for (int j = 0; j < Nc; ++j) A[(size_t)i * Nc + j] += wi * phi[j];
              for (int a = 0; a < 3; ++a) B[(size_t)i * 3 + a] += wi * uold[((size_t)e * npts + q) * 3 + a];
            }
          }
      if (solve_dense(Nc, A, B, 3) != 0) {
#pragma omp atomic write
        status = -1;
        continue;
      }
      for (int a = 0; a < 3; ++a) {
        double *uc = u_new + ((size_t)c * 3 + a) * n3;
        for (int i = 0; i < n3; ++i) uc[i] = B[(size_t)i * 3 + a];
        double *ue = u_new + 3L * M->np + ((size_t)e * 3 + a) * nef;
        for (int v = 0; v < nef; ++v) ue[v] = Nc == N ? B[(size_t)(n3 + v) * 3 + a] : 0.0;
      }
    }
    free(A); free(B); free(phi);
    ptab_free(&t);
  }
  free(uold);
  return status;
}

/* ----------------------------------------------------------------------------------------------
 * Pressure gradient (Sec. 4.2): y = P(v, p) = -(div v, p)_K + (v, {{p}} n)_dK for every velocity
 * test function (standard and enriched), {{p}} = p^- on walls (projection step, eq.
 * projectionspat). Point sets as the divergence.
 * ---------------------------------------------------------------------------------------------- */
static double eval_p(const omesh *M, const double *p, int c, const ptab *t) {
  const double *pc = p + (size_t)c * t->n3;
  double v = 0.0;
  for (int i = 0; i < t->n3; ++i) v += t->phi[i] * pc[i];
  return v;
}

int dgo_gradient(void *h, const double *p, double *y) {
  omesh *M = (omesh *)h;
  int n3 = M->n1 * M->n1 * M->n1;
  memset(y, 0, sizeof(double) * M->nu);
#pragma omp parallel
  {
    ptab t, tn; ptab_alloc(&t, M); ptab_alloc(&tn, M);
    double gx[MAXP], gw[MAXP], gy[MAXP], gwy[MAXP], gx2[MAXP], gw2[MAXP];
#pragma omp for schedule(dynamic, 4)
    for (int c = 0; c < M->nc; ++c) {
      int nq[3];
      cell_points(M, c, OP_LINEAR, nq);
      dgo_gauss(nq[0], gx, gw); dgo_gauss(nq[1], gy, gwy);
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0) {
            double xi[3] = {gx[q0], gy[q1], gx[q2]};
            tabulate(M, c, xi, &t);
            double dV = fabs(t.detJ) * gw[q0] * gwy[q1] * gw[q2];
            double pv = eval_p(M, p, c, &t);
            for (int a = 0; a < 3; ++a) {
              double *yc = y + ((size_t)c * 3 + a) * n3;
              for (int i = 0; i < n3; ++i) yc[i] -= dV * t.gphi[3 * i + a] * pv;
              if (t.enriched) {
                double *ye = y + 3L * M->np + ((size_t)M->enr[c] * 3 + a) * M->nef;
                for (int v = 0; v < M->nef; ++v) ye[v] -= dV * t.egphi[v][a] * pv;
              }
            }
          }
      for (int f = 0; f < 6; ++f) {
        int nb = neighbour(M, c, f);
        int d = f / 2, side = f % 2, t1, t2, m1, m2;
        face_points(M, c, nb, d, OP_LINEAR, &t1, &t2, &m1, &m2);
        dgo_gauss(m1, gx, gw); dgo_gauss(m2, gx2, gw2);
        for (int bq = 0; bq < m2; ++bq)
          for (int a1 = 0; a1 < m1; ++a1) {
            double xi[3], xn[3], n[3];
            xi[d] = side; xi[t1] = gx[a1]; xi[t2] = gx2[bq];
            tabulate(M, c, xi, &t);
            double dA = face_geom(t.Ji, t.detJ, d, side, n) * gw[a1] * gw2[bq];
            double pm = eval_p(M, p, c, &t), avg = pm;
            if (nb >= 0) {
              xn[d] = 1 - side; xn[t1] = gx[a1]; xn[t2] = gx2[bq];
              tabulate(M, nb, xn, &tn);
              avg = 0.5 * (pm + eval_p(M, p, nb, &tn));
            }
            for (int a = 0; a < 3; ++a) {
              double *yc = y + ((size_t)c * 3 + a) * n3, fa = dA * avg * n[a];
              for (int i = 0; i < n3; ++i) yc[i] += t.phi[i] * fa;
              if (t.enriched) {
                double *ye = y + 3L * M->np + ((size_t)M->enr[c] * 3 + a) * M->nef;
                for (int v = 0; v < M->nef; ++v) ye[v] += t.ephi[v] * fa;
              }
            }
          }
      }
    }
    ptab_free(&t); ptab_free(&tn);
  }
  return 0;
}

/* ----------------------------------------------------------------------------------------------
 * Div-div penalty (Sec. 4.2, eq. div-div): y = D(v, u) = (div v, tau_D div u)_K with a constant
 * tau_D per cell (eq. tauD: |u^n|_K h dt / Cr, computed by dgo_tau_divdiv). Cell-local.
 * ---------------------------------------------------------------------------------------------- */
int dgo_divdiv(void *h, const double *tau_d, const double *u, double *y) {
  omesh *M = (omesh *)h;
  int n3 = M->n1 * M->n1 * M->n1;
  memset(y, 0, sizeof(double) * M->nu);
#pragma omp parallel
  {
    ptab t; ptab_alloc(&t, M);
    double gx[MAXP], gw[MAXP], gy[MAXP], gwy[MAXP];
#pragma omp for schedule(dynamic, 4)
    for (int c = 0; c < M->nc; ++c) {
      int nq[3];
      cell_points(M, c, OP_LINEAR, nq);
      dgo_gauss(nq[0], gx, gw); dgo_gauss(nq[1], gy, gwy);
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0) {
            double xi[3] = {gx[q0], gy[q1], gx[q2]};
            tabulate(M, c, xi, &t);
            double dV = fabs(t.detJ) * gw[q0] * gwy[q1] * gw[q2];
            vstate s; eval_vel(M, u, c, &t, &s);
            double dv = 0.0;
            for (int a = 0; a < 3; ++a) dv += s.gb[a][a] + s.gt[a][a];
            double f = dV * tau_d[c] * dv;
            for (int a = 0; a < 3; ++a) {
              double *yc = y + ((size_t)c * 3 + a) * n3;
              for (int i = 0; i < n3; ++i) yc[i] += t.gphi[3 * i + a] * f;
              if (t.enriched) {
                double *ye = y + 3L * M->np + ((size_t)M->enr[c] * 3 + a) * M->nef;
                for (int v = 0; v < M->nef; ++v) ye[v] += t.egphi[v][a] * f;
              }
            }
          }
    }
    ptab_free(&t);
  }
  return 0;
}

/* tau_D per cell (eq. tauD): the volume average of |u| over the cell times h dt / Cr, with h the cube
 * root of the cell volume. */
/* Rate of the adaptive time step (Sec. 4.1: the step is chosen from a CFL condition with the
 * Courant number Cr; the condition itself is not restated there, reading in the design notes): the
 * largest Euclidean norm of J^-1 (ubar + u~), the velocity in reference-cell lengths per unit time,
 * over the volume points of the linear point set of every cell (k+1 Gauss points per direction, q_w
 * wall-normal in enriched cells). The step is then Cr / (k^1.5 rate). */
double dgo_cfl_rate(void *h, const double *u) {
  omesh *M = (omesh *)h;
  double best = 0.0;
#pragma omp parallel
  {
    ptab t; ptab_alloc(&t, M);
    double gx[MAXP], gw[MAXP], gy[MAXP], gwy[MAXP];
    double mine = 0.0;
#pragma omp for schedule(dynamic, 4)
    for (int c = 0; c < M->nc; ++c) {
      int nq[3];
      cell_points(M, c, OP_LINEAR, nq);
      dgo_gauss(nq[0], gx, gw); dgo_gauss(nq[1], gy, gwy);
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0) {
            double xi[3] = {gx[q0], gy[q1], gx[q2]};
            tabulate(M, c, xi, &t);
            vstate sv; eval_vel(M, u, c, &t, &sv);
            double uu[3] = {sv.ub[0] + sv.ut[0], sv.ub[1] + sv.ut[1], sv.ub[2] + sv.ut[2]};
            double r2 = 0.0;
            for (int r = 0; r < 3; ++r) {
              double w = t.Ji[r][0] * uu[0] + t.Ji[r][1] * uu[1] + t.Ji[r][2] * uu[2];
              r2 += w * w;
            }
            if (sqrt(r2) > mine) mine = sqrt(r2);
          }
    }
#pragma omp critical
    if (mine > best) best = mine;
    ptab_free(&t);
  }
  return best;
}

int dgo_tau_divdiv(void *h, const double *u, double dt, double cr, double *tau_d) {
  omesh *M = (omesh *)h;
#pragma omp parallel
  {
    ptab t; ptab_alloc(&t, M);
    double gx[MAXP], gw[MAXP], gy[MAXP], gwy[MAXP];
#pragma omp for schedule(dynamic, 4)
    for (int c = 0; c < M->nc; ++c) {
      int nq[3];
      cell_points(M, c, OP_LINEAR, nq);
      dgo_gauss(nq[0], gx, gw); dgo_gauss(nq[1], gy, gwy);
      double vol = 0.0, mag = 0.0;
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0) {
            double xi[3] = {gx[q0], gy[q1], gx[q2]};
            tabulate(M, c, xi, &t);
            double dV = fabs(t.detJ) * gw[q0] * gwy[q1] * gw[q2];
            vstate s; eval_vel(M, u, c, &t, &s);
            double uu[3] = {s.ub[0] + s.ut[0], s.ub[1] + s.ut[1], s.ub[2] + s.ut[2]};
            vol += dV;
            mag += dV * sqrt(uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]);
          }
      tau_d[c] = (mag / vol) * cbrt(vol) * dt / cr;
    }
    ptab_free(&t);
  }
  return 0;
}

/* ----------------------------------------------------------------------------------------------
 * Inverse of the velocity mass matrix (Sec. 4.2 mass term; the explicit convective step needs
 * M^-1 exactly): cell by cell, the mass matrix of the cell's space (standard plus switched-on
 * enrichment) assembled with its velocity point set and solved by Gaussian elimination with
 * partial pivoting. x = M^-1 r; switched-off enrichment slots are zero.
 * ---------------------------------------------------------------------------------------------- */
int dgo_inverse_mass(void *h, const double *r, double *x) {
  omesh *M = (omesh *)h;
  const int n3 = M->n1 * M->n1 * M->n1, nef = M->nef, N = n3 + nef;
  memset(x, 0, sizeof(double) * M->nu);
  int status = 0;
#pragma omp parallel
  {
    ptab t; ptab_alloc(&t, M);
    double gx[MAXP], gw[MAXP], gy[MAXP], gwy[MAXP];
    double *A = (double *)malloc(sizeof(double) * (size_t)N * N);
    double *B = (double *)malloc(sizeof(double) * (size_t)N * 3);
#pragma omp for schedule(dynamic, 2)
    for (int c = 0; c < M->nc; ++c) {
      int nq[3], en = M->enr[c];
      const int Nc = en >= 0 ? N : n3;
      cell_points(M, c, OP_LINEAR, nq);
      dgo_gauss(nq[0], gx, gw); dgo_gauss(nq[1], gy, gwy);
      memset(A, 0, sizeof(double) * (size_t)N * N);
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0) {
            double xi[3] = {gx[q0], gy[q1], gx[q2]}, phi[8 + MAXP * MAXP * MAXP];
            tabulate(M, c, xi, &t);
            double dV = fabs(t.detJ) * gw[q0] * gwy[q1] * gw[q2];
            for (int i = 0; i < n3; ++i) phi[i] = t.phi[i];
            for (int v = 0; v < nef && en >= 0; ++v) phi[n3 + v] = t.ephi[v];
            for (int i = 0; i < Nc; ++i)
              for (int j = 0; j < Nc; ++j) A[(size_t)i * Nc + j] += dV * phi[i] * phi[j];
          }
      for (int a = 0; a < 3; ++a) {
        for (int i = 0; i < n3; ++i) B[(size_t)i * 3 + a] = r[((size_t)c * 3 + a) * n3 + i];
        for (int v = 0; v < nef && en >= 0; ++v) B[(size_t)(n3 + v) * 3 + a] = r[3L * M->np + ((size_t)en * 3 + a) * nef + v];
      }
      if (solve_dense(Nc, A, B, 3) != 0) {
#pragma omp atomic write
        status = -1;
        continue;
      }
      for (int a = 0; a < 3; ++a) {
        for (int i = 0; i < n3; ++i) x[((size_t)c * 3 + a) * n3 + i] = B[(size_t)i * 3 + a];
        for (int v = 0; v < nef && en >= 0; ++v) x[3L * M->np + ((size_t)en * 3 + a) * nef + v] = B[(size_t)(n3 + v) * 3 + a];
      }
    }
    free(A); free(B);
    ptab_free(&t);
  }
  return status;
}

/* ----------------------------------------------------------------------------------------------
 * Vorticity and the high-order pressure Neumann data (Sec. 4.1 eq. bc_d_pres, Sec. 4.2 ipflux).
 * dgo_curl: y = (v, curl u)_K for every velocity test function (the right-hand side of the L2
 * projection omega_h = M^-1 y). dgo_pressure_neumann: adds to a pressure vector the wall integrals
 * (q, g) with g = -(sum_i beta_i (div(u^{n-i} x u^{n-i}) + nu curl omega^{n-i}) - f) . n, evaluated
 * with the interior traces (k+1 Gauss points per tangential direction, as the Laplace faces).
 * ---------------------------------------------------------------------------------------------- */
int dgo_curl(void *h, const double *u, double *y) {
  omesh *M = (omesh *)h;
  int n3 = M->n1 * M->n1 * M->n1;
  memset(y, 0, sizeof(double) * M->nu);
#pragma omp parallel
  {
    ptab t; ptab_alloc(&t, M);
    double gx[MAXP], gw[MAXP], gy[MAXP], gwy[MAXP];
#pragma omp for schedule(dynamic, 4)
    for (int c = 0; c < M->nc; ++c) {
      int nq[3];
      cell_points(M, c, OP_LINEAR, nq);
      dgo_gauss(nq[0], gx, gw); dgo_gauss(nq[1], gy, gwy);
      for (int q2 = 0; q2 < nq[2]; ++q2)
        for (int q1 = 0; q1 < nq[1]; ++q1)
          for (int q0 = 0; q0 < nq[0]; ++q0) {
            double xi[3] = {gx[q0], gy[q1], gx[q2]};
            tabulate(M, c, xi, &t);
            double dV = fabs(t.detJ) * gw[q0] * gwy[q1] * gw[q2];
            vstate s; eval_vel(M, u, c, &t, &s);
            double G[3][3];
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) G[a][b] = s.gb[a][b] + s.gt[a][b];
            double w[3] = {G[2][1] - G[1][2], G[0][2] - G[2][0], G[1][0] - G[0][1]};
            for (int a = 0; a < 3; ++a) {
              double *yc = y + ((size_t)c * 3 + a) * n3;
              for (int i = 0; i < n3; ++i) yc[i] += dV * t.phi[i] * w[a];
              if (t.enriched) {
                double *ye = y + 3L * M->np + ((size_t)M->enr[c] * 3 + a) * M->nef;
                for (int v = 0; v < M->nef; ++v) ye[v] += dV * t.ephi[v] * w[a];
              }
            }
          }
    }
    ptab_free(&t);
  }
  return 0;
}

int dgo_pressure_neumann(void *h, const double *u0, const double *u1, const double *w0, const double *w1, double b0,
                         double b1, const double *f, double *y) {
  omesh *M = (omesh *)h;
  const int nx = M->P.nx, ny = M->P.ny, nz = M->P.nz, n1 = M->n1, n3 = n1 * n1 * n1;
  double gx[MAXP], gw[MAXP];
  ptab t; ptab_alloc(&t, M);
  const double *us[2] = {u0, u1}, *ws[2] = {w0, w1};
  const double bs[2] = {b0, b1};
  for (int wall = 0; wall < 2; ++wall)
    for (int kz = 0; kz < nz; ++kz)
      for (int i = 0; i < nx; ++i) {
        const int j = wall ? ny - 1 : 0, c = cell_id(M, i, j, kz);
        double *yc = y + (size_t)c * n3;
        const int nf = (M->P.full_q && M->enr[c] >= 0) ? M->P.q_wall : n1;
        dgo_gauss(nf, gx, gw);
        for (int q2 = 0; q2 < nf; ++q2)
          for (int q0 = 0; q0 < nf; ++q0) {
            double xi[3] = {gx[q0], wall ? 1.0 : 0.0, gx[q2]}, nrm[3];
            tabulate(M, c, xi, &t);
            double dA = face_geom(t.Ji, t.detJ, 1, wall, nrm) * gw[q0] * gw[q2];
            double acc[3] = {-f[0], -f[1], -f[2]};
            for (int h2 = 0; h2 < 2; ++h2) {
              if (bs[h2] == 0.0 || !us[h2]) continue;
              vstate s; eval_vel(M, us[h2], c, &t, &s);
              vstate so; eval_vel(M, ws[h2], c, &t, &so);
              double U[3], G[3][3], GW[3][3];
              for (int a = 0; a < 3; ++a) {
                U[a] = s.ub[a] + s.ut[a];
                for (int b = 0; b < 3; ++b) {
                  G[a][b] = s.gb[a][b] + s.gt[a][b];
                  GW[a][b] = so.gb[a][b] + so.gt[a][b];
                }
              }
              double dv = G[0][0] + G[1][1] + G[2][2];
              double cw[3] = {GW[2][1] - GW[1][2], GW[0][2] - GW[2][0], GW[1][0] - GW[0][1]};
              for (int a = 0; a < 3; ++a) {
                double conv = U[a] * dv;
                for (int b = 0; b < 3; ++b) conv += U[b] * G[a][b];
                acc[a] += bs[h2] * (conv + M->P.nu * cw[a]);
              }
            }
            double g = -(acc[0] * nrm[0] + acc[1] * nrm[1] + acc[2] * nrm[2]);
            for (int q = 0; q < n3; ++q) yc[q] += dA * t.phi[q] * g;
          }
      }
  ptab_free(&t);
  return 0;
}
