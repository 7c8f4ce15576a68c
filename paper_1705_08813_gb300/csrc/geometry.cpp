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
