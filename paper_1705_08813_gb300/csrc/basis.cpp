// Host-side 1-D rules and basis tables of the library (Sec. 4.4: Gauss quadrature with k+1 or
// floor(3k/2)+1 points; nodal Lagrange basis on the k+1 Gauss-Lobatto points).
#include <cmath>
#include <cstring>

#include "dgw_internal.h"

namespace dgw {

// Legendre recursion returning P_m(t) and P_{m-1}(t).
static void legendre_pair(int m, double t, double &pm, double &pm1) {
  double a = 1.0, b = t;   // P_0, P_1
  if (m == 0) { pm = 1.0; pm1 = 0.0; return; }
  for (int j = 1; j < m; ++j) {
    double c = ((2 * j + 1) * t * b - j * a) / (j + 1);
    a = b; b = c;
  }
  pm = b; pm1 = a;
}

// n-point Gauss-Legendre rule mapped to [0,1] (ascending). Newton from Tricomi's estimate.
void gauss_rule(int n, double *x, double *w) {
  for (int i = 1; i <= n; ++i) {
    double t = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * std::cos(M_PI * (4.0 * i - 1.0) / (4.0 * n + 2.0));
    double dp = 1.0;
    for (int it = 0; it < 64; ++it) {
      double p, p1;
      legendre_pair(n, t, p, p1);
      dp = n * (p1 - t * p) / (1.0 - t * t);
      double step = p / dp;
      t -= step;
      if (std::fabs(step) <= 4e-17) break;
    }
    double p, p1;
    legendre_pair(n, t, p, p1);
    dp = n * (p1 - t * p) / (1.0 - t * t);
    x[n - i] = 0.5 * (t + 1.0);
    w[n - i] = 1.0 / ((1.0 - t * t) * dp * dp);
  }
}

// n Gauss-Lobatto points on [0,1]: endpoints plus the zeros of P'_{n-1}, found by Newton on
// (1-t^2) P'_{n-1}(t) = (n-1) (P_{n-2} - t P_{n-1}).
void lobatto_nodes(int n, double *x) {
  x[0] = 0.0;
  x[n - 1] = 1.0;
  const int m = n - 1;
  for (int i = 1; i < m; ++i) {
    double t = std::cos(M_PI * (m - i) / m);   // ascending initial guesses
    for (int it = 0; it < 64; ++it) {
      double p, p1;
      legendre_pair(m, t, p, p1);
      double g = m * (p1 - t * p);                      // (1-t^2) P'_m
      // d/dt [(1-t^2) P'_m] = -m(m+1) P_m (Legendre ODE)
      double dg = -m * (m + 1.0) * p;
      double step = g / dg;
      t -= step;
      if (std::fabs(step) <= 4e-17) break;
    }
    x[i] = 0.5 * (t + 1.0);
  }
}

// Barycentric Lagrange basis on nodes z[0..n-1]: values l_j(s) and derivatives l_j'(s).
void lagrange_row(int n, const double *z, double s, double *val, double *der) {
  double bw[NMAX];
  for (int j = 0; j < n; ++j) {
    double p = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) p *= (z[j] - z[m]);
    bw[j] = 1.0 / p;
  }
  // value: l_j(s) = bw_j prod_{m!=j} (s - z_m); derivative by the product rule
  for (int j = 0; j < n; ++j) {
    double v = bw[j], d = 0.0;
    for (int m = 0; m < n; ++m) {
      if (m == j) continue;
      d = d * (s - z[m]) + v;
      v *= (s - z[m]);
    }
    val[j] = v;
    der[j] = d;
  }
}

template <typename T>
void fill_basis(int k, int q_conv, int q_wall, Basis<T> *b) {
  std::memset(b, 0, sizeof(*b));
  const int n = k + 1;
  b->n1 = n;
  b->q[QSET_LIN] = n;
  b->q[QSET_CONV] = q_conv;
  b->q[QSET_WALL] = q_wall;
  double z[NMAX];
  lobatto_nodes(n, z);
  for (int s = 0; s < NQSET; ++s) {
    double x[QMAX], w[QMAX];
    gauss_rule(b->q[s], x, w);
    for (int q = 0; q < b->q[s]; ++q) {
      double v[NMAX], d[NMAX];
      lagrange_row(n, z, x[q], v, d);
      for (int j = 0; j < n; ++j) {
        b->S[s][q * n + j] = (T)v[j];
        b->D[s][q * n + j] = (T)d[j];
      }
      b->x[s][q] = (T)x[q];
      b->w[s][q] = (T)w[q];
    }
  }
  for (int side = 0; side < 2; ++side) {
    double v[NMAX], d[NMAX];
    lagrange_row(n, z, (double)side, v, d);
    for (int j = 0; j < n; ++j) b->dend[side][j] = (T)d[j];
  }
  for (int a = 0; a < n; ++a)
    for (int c = 0; c < n; ++c) {
      double s = 0.0;
      for (int q = 0; q < b->q[QSET_LIN]; ++q) s += (double)b->w[QSET_LIN][q] * b->S[QSET_LIN][q * n + a] * b->S[QSET_LIN][q * n + c];
      b->mass[a * n + c] = (T)s;
    }
  for (int o = 0; o < 2; ++o)
    for (int i = 0; i < n; ++i) {
      double v[NMAX], d[NMAX];
      lagrange_row(n, z, 0.5 * (o + z[i]), v, d);
      for (int j = 0; j < n; ++j) b->P[o][i * n + j] = (T)v[j];
    }
}

// P[i*n + j] = l_j(a + b z_i): nodal embedding of the parent cell's basis into a child whose local
// coordinate x maps to a + b x in the parent (z: Gauss-Lobatto nodes).
void embed_matrix(int n, double a, double b, double *P) {
  double z[NMAX];
  lobatto_nodes(n, z);
  for (int i = 0; i < n; ++i) {
    double v[NMAX], d[NMAX];
    lagrange_row(n, z, a + b * z[i], v, d);
    for (int j = 0; j < n; ++j) P[i * n + j] = v[j];
  }
}

template void fill_basis<double>(int, int, int, Basis<double> *);
template void fill_basis<float>(int, int, int, Basis<float> *);

}  // namespace dgw
