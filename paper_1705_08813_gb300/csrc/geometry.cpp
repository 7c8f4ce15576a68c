// Host geometry of the channel of boxes: row heights, penalty parameters and the Jacobi
// diagonal of the SIPG Laplacian (used by the fine mesh and by every multigrid level).
#include <algorithm>
#include <cmath>

#include "dgw_internal.h"

namespace dgw {

void box_geometry(int k, int nx, int ny, int nz, double lx, double lz, const std::vector<double> &yv, BoxGeometry &g) {
  g.nx = nx; g.ny = ny; g.nz = nz; g.k = k;
  g.hx = lx / nx;
  g.hz = lz / nz;
  g.yv = yv;
  g.hy.resize(ny);
  for (int j = 0; j < ny; ++j) g.hy[j] = yv[j + 1] - yv[j];
  const int n = k + 1;
  g.tau.resize((size_t)nx * ny * nz);
  for (int kz = 0; kz < nz; ++kz)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const double hy = g.hy[j];
        const double wb = j == 0 ? 1.0 : 0.5, wt = j == ny - 1 ? 1.0 : 0.5;
        const double A = hy * g.hz + g.hx * hy + g.hx * g.hz * (wb + wt);
        g.tau[i + (size_t)nx * (j + (size_t)ny * kz)] = (double)(n * n) * A / (g.hx * hy * g.hz);
      }
}

void laplace_diagonal(const BoxGeometry &g, const Basis<double> &B, std::vector<double> &dg) {
  const int n = g.k + 1, nx = g.nx, ny = g.ny, nz = g.nz;
  const int q = B.q[QSET_LIN];
  std::vector<double> m1(n, 0.0), k1(n, 0.0);
  for (int a = 0; a < n; ++a)
    for (int t = 0; t < q; ++t) {
      m1[a] += B.w[QSET_LIN][t] * B.S[QSET_LIN][t * n + a] * B.S[QSET_LIN][t * n + a];
      k1[a] += B.w[QSET_LIN][t] * B.D[QSET_LIN][t * n + a] * B.D[QSET_LIN][t * n + a];
    }
  dg.assign((size_t)nx * ny * nz * n * n * n, 0.0);
  for (int kz = 0; kz < nz; ++kz)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const int c = i + nx * (j + ny * kz);
        const double h[3] = {g.hx, g.hy[j], g.hz};
        const double vol = h[0] * h[1] * h[2];
        for (int i2 = 0; i2 < n; ++i2)
          for (int i1 = 0; i1 < n; ++i1)
            for (int i0 = 0; i0 < n; ++i0) {
              const int id[3] = {i0, i1, i2};
              double v = vol * (k1[i0] * m1[i1] * m1[i2] / (h[0] * h[0]) + m1[i0] * k1[i1] * m1[i2] / (h[1] * h[1]) +
                                m1[i0] * m1[i1] * k1[i2] / (h[2] * h[2]));
              for (int f = 0; f < 6; ++f) {
                const int d = f >> 1, side = f & 1;
                int ii = i, jj = j, kk = kz;
                const int s = side ? 1 : -1;
                if (d == 0) ii = (i + s + nx) % nx;
                else if (d == 2) kk = (kz + s + nz) % nz;
                else { jj = j + s; if (jj < 0 || jj >= ny) continue; }
                const int nb = ii + nx * (jj + ny * kk);
                const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
                const double sgn = side ? 1.0 : -1.0;
                const double tau = std::max(g.tau[c], g.tau[nb]);
                const double area = h[t1] * h[t2] * m1[id[t1]] * m1[id[t2]];
                const int Ls = side ? n - 1 : 0, Lo = side ? 0 : n - 1;
                const double ps = id[d] == Ls ? 1.0 : 0.0;
                const double dns = sgn / h[d] * B.dend[side][id[d]];
                double po = 0.0, dno = 0.0;
                if (nb == c) {   // a single cell across a periodic direction
                  po = id[d] == Lo ? 1.0 : 0.0;
                  dno = sgn / h[d] * B.dend[1 - side][id[d]];
                }
                const double jump = ps - po;
                v -= area * (0.5 * dns * jump + ps * (0.5 * (dns + dno) - tau * jump));
              }
              dg[(size_t)c * n * n * n + i0 + n * (i1 + n * i2)] = v;
            }
      }
}

}  // namespace dgw

// ------------------------------------------------------------------------------------------------
// Curved bump channel (geometry 1). The lower wall follows y_w(x) = 0.3 cos^2(pi (x - lx/2) / 2) for
// |x - lx/2| < 1 (0 elsewhere), the upper wall is y = ly, and the rows between them are graded by
// the tanh map of Sec. 5.1 in the logical coordinate. Cells are isoparametric Q_k images of the
// reference cube: their Gauss-Lobatto nodes are points of the map and J is the derivative of the
// Lagrange interpolant of those nodes (Sec. 5.2: the periodic-hill mesh is mapped onto the exact
// geometry with the same polynomial ansatz as the solution). The map is an extrusion along z, so
// J at a point depends on (i, j, xi_0, xi_1) only and the tables are kept per column (i, j).

namespace dgw {

static double bump_wall_height(double lx, double x) {
  const double s = x - 0.5 * lx;
  if (std::fabs(s) < 1.0) {
    const double c = std::cos(M_PI * s / 2.0);
    return 0.3 * c * c;
  }
  return 0.0;
}

void bump_point(const dgw_mesh_params &P, int nx, int ny, double a0, double a1, double *x, double *y) {
  const double xx = P.lx * a0 / nx;
  const double yw = bump_wall_height(P.lx, xx);
  const double f = std::tanh(P.stretch_gamma * (2.0 * a1 / ny - 1.0)) / std::tanh(P.stretch_gamma);
  *x = xx;
  *y = yw + (P.ly - yw) * 0.5 * (1.0 + f);
}

// J^-1 (row-major) and det J of the interpolated map at (xi0, xi1) of a column with nodal
// positions X, Y (index a + n*b) and z-spacing hz.
static void column_metric(int n, const double *z, const double *X, const double *Y, double hz, double xi0, double xi1,
                          double *rec) {
  double l0[NMAX], d0[NMAX], l1[NMAX], d1[NMAX];
  lagrange_row(n, z, xi0, l0, d0);
  lagrange_row(n, z, xi1, l1, d1);
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, hz}};
  for (int b = 0; b < n; ++b)
    for (int a = 0; a < n; ++a) {
      const double gx = d0[a] * l1[b], gy = l0[a] * d1[b];
      J[0][0] += gx * X[a + n * b];
      J[0][1] += gy * X[a + n * b];
      J[1][0] += gx * Y[a + n * b];
      J[1][1] += gy * Y[a + n * b];
    }
  // inverse by cofactors
  const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1], c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2],
               c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  rec[0] = c00 / det;
  rec[1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  rec[2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  rec[3] = c01 / det;
  rec[4] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  rec[5] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  rec[6] = c02 / det;
  rec[7] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  rec[8] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  rec[9] = det;
}

void curved_geometry(const dgw_mesh_params &P, int nx, int ny, int nz, int k, const Basis<double> &B, CurvedHost &G) {
  G.nx = nx; G.ny = ny; G.nz = nz; G.k = k;
  const int n = k + 1, ncol = nx * ny;
  const double hz = P.lz / nz;
  double z[NMAX];
  lobatto_nodes(n, z);
  G.xn.assign((size_t)ncol * n * n, 0.0);
  G.yn.assign((size_t)ncol * n * n, 0.0);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
          const size_t o = (size_t)(i + nx * j) * n * n + a + n * b;
          bump_point(P, nx, ny, i + z[a], j + z[b], &G.xn[o], &G.yn[o]);
        }
  const int xsets[2] = {QSET_LIN, QSET_CONV};
  const bool fq = P.full_quadrature != 0;   // the q_w^3 rule needs the wall set along x as well
  for (int pair = 0; pair < NMVOL; ++pair) {
    if (pair == MVOL_WALL_WALL && !fq) continue;
    const int sx = pair == MVOL_WALL_WALL ? QSET_WALL : xsets[pair & 1];
    const int sy = (pair & 2) || pair == MVOL_WALL_WALL ? QSET_WALL : sx;
    const int qx = B.q[sx], qy = B.q[sy];
    G.mvol[pair].assign((size_t)ncol * qx * qy * MREC, 0.0);
    for (int m = 0; m < ncol; ++m)
      for (int a1 = 0; a1 < qy; ++a1)
        for (int a0 = 0; a0 < qx; ++a0)
          column_metric(n, z, &G.xn[(size_t)m * n * n], &G.yn[(size_t)m * n * n], hz, B.x[sx][a0], B.x[sy][a1],
                        &G.mvol[pair][((size_t)m * qx * qy + a0 + qx * a1) * MREC]);
  }
  for (int set = 0; set < NQSET; ++set) {
    const int q = B.q[set];
    G.mxf[set].assign((size_t)ncol * 2 * q * MREC, 0.0);
    for (int m = 0; m < ncol; ++m)
      for (int side = 0; side < 2; ++side)
        for (int a = 0; a < q; ++a)
          column_metric(n, z, &G.xn[(size_t)m * n * n], &G.yn[(size_t)m * n * n], hz, (double)side, B.x[set][a],
                        &G.mxf[set][(((size_t)m * 2 + side) * q + a) * MREC]);
  }
  for (int set = 0; set < NQSET; ++set) {
    if (set == QSET_WALL && !fq) continue;
    const int q = B.q[set];
    G.myf[set].assign((size_t)ncol * 2 * q * MREC, 0.0);
    for (int m = 0; m < ncol; ++m)
      for (int side = 0; side < 2; ++side)
        for (int a = 0; a < q; ++a)
          column_metric(n, z, &G.xn[(size_t)m * n * n], &G.yn[(size_t)m * n * n], hz, B.x[set][a], (double)side,
                        &G.myf[set][(((size_t)m * 2 + side) * q + a) * MREC]);
  }
  // penalty tau_IP = (k+1)^2 A/V with (k+2)-point Gauss integration of the curved cell (interior
  // faces weighted 1/2, wall faces 1)
  const int nq = n + 1;
  double gx[NMAX + 2], gw[NMAX + 2];
  gauss_rule(nq, gx, gw);
  G.tau.assign(ncol, 0.0);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const int m = i + nx * j;
      const double *X = &G.xn[(size_t)m * n * n], *Y = &G.yn[(size_t)m * n * n];
      auto grad_norm = [](const double *rec, int d) {
        return std::sqrt(rec[d * 3] * rec[d * 3] + rec[d * 3 + 1] * rec[d * 3 + 1] + rec[d * 3 + 2] * rec[d * 3 + 2]);
      };
      double V = 0.0, A = 0.0, rec[MREC];
      for (int q1 = 0; q1 < nq; ++q1)
        for (int q0 = 0; q0 < nq; ++q0) {
          column_metric(n, z, X, Y, hz, gx[q0], gx[q1], rec);
          // volume (the z weights sum to one) and the two faces xi_2 = 0, 1
          V += std::fabs(rec[9]) * gw[q0] * gw[q1];
          A += 2 * 0.5 * std::fabs(rec[9]) * grad_norm(rec, 2) * gw[q0] * gw[q1];
        }
      for (int side = 0; side < 2; ++side)
        for (int q = 0; q < nq; ++q) {
          column_metric(n, z, X, Y, hz, (double)side, gx[q], rec);   // faces xi_0 = side
          A += 0.5 * std::fabs(rec[9]) * grad_norm(rec, 0) * gw[q];
          column_metric(n, z, X, Y, hz, gx[q], (double)side, rec);   // faces xi_1 = side
          const bool wall = (side == 0 && j == 0) || (side == 1 && j == ny - 1);
          A += (wall ? 1.0 : 0.5) * std::fabs(rec[9]) * grad_norm(rec, 1) * gw[q];
        }
      G.tau[m] = (double)(n * n) * A / V;
    }
  // SIPG Laplacian tables at the k+1 Gauss points (QSET_LIN)
  const int q = B.q[QSET_LIN];
  const double *w = B.w[QSET_LIN];
  G.lvol.assign((size_t)ncol * q * q * q * 6, 0.0);
  G.lface.assign((size_t)ncol * 6 * q * q * 7, 0.0);
  for (int m = 0; m < ncol; ++m)
    for (int a2 = 0; a2 < q; ++a2)
      for (int a1 = 0; a1 < q; ++a1)
        for (int a0 = 0; a0 < q; ++a0) {
          const double *r = &G.mvol[0][((size_t)m * q * q + a0 + q * a1) * MREC];
          const double dv = std::fabs(r[9]) * w[a0] * w[a1] * w[a2];
          auto jj = [&](int x, int y) { return dv * (r[x * 3] * r[y * 3] + r[x * 3 + 1] * r[y * 3 + 1] + r[x * 3 + 2] * r[y * 3 + 2]); };
          double *o = &G.lvol[((size_t)m * q * q * q + a0 + q * (a1 + q * a2)) * 6];
          o[0] = jj(0, 0); o[1] = jj(1, 1); o[2] = jj(2, 2); o[3] = jj(0, 1); o[4] = jj(0, 2); o[5] = jj(1, 2);
        }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const int m = i + nx * j;
      for (int f = 0; f < 6; ++f) {
        const int d = f >> 1, s = f & 1;
        int mo = m;
        if (d == 0) mo = ((i + (s ? 1 : -1) + nx) % nx) + nx * j;
        if (d == 1) {
          const int jn = j + (s ? 1 : -1);
          if (jn < 0 || jn >= ny) continue;   // homogeneous Neumann wall: no face terms
          mo = i + nx * jn;
        }
        for (int a2 = 0; a2 < q; ++a2)
          for (int a1 = 0; a1 < q; ++a1) {
            const double *rs, *ro;
            if (d == 0) {
              rs = &G.mxf[QSET_LIN][(((size_t)m * 2 + s) * q + a1) * MREC];
              ro = &G.mxf[QSET_LIN][(((size_t)mo * 2 + 1 - s) * q + a1) * MREC];
            } else if (d == 1) {
              rs = &G.myf[QSET_LIN][(((size_t)m * 2 + s) * q + a1) * MREC];
              ro = &G.myf[QSET_LIN][(((size_t)mo * 2 + 1 - s) * q + a1) * MREC];
            } else {
              rs = ro = &G.mvol[0][((size_t)m * q * q + a1 + q * a2) * MREC];
            }
            const double sg = s ? 1.0 : -1.0;
            const double nrm = std::sqrt(rs[d * 3] * rs[d * 3] + rs[d * 3 + 1] * rs[d * 3 + 1] + rs[d * 3 + 2] * rs[d * 3 + 2]);
            const double nv[3] = {sg * rs[d * 3] / nrm, sg * rs[d * 3 + 1] / nrm, sg * rs[d * 3 + 2] / nrm};
            const double dA = std::fabs(rs[9]) * nrm * w[a1] * w[a2];
            double *o = &G.lface[(((size_t)m * 6 + f) * q * q + a1 + q * a2) * 7];
            o[0] = dA;
            for (int r = 0; r < 3; ++r) {
              o[1 + r] = dA * (rs[r * 3] * nv[0] + rs[r * 3 + 1] * nv[1] + rs[r * 3 + 2] * nv[2]);
              o[4 + r] = dA * (ro[r * 3] * nv[0] + ro[r * 3 + 1] * nv[1] + ro[r * 3 + 2] * nv[2]);
            }
          }
      }
    }
}

}  // namespace dgw
