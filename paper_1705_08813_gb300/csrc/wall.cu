// Wall tables and eddy viscosity of the enriched cells.
//
// Sec. 3.2: the wall distance y_h and the wall shear stress tau_w,h are interpolated with the
// linear C0 functions of the cell's vertices; y+ = y_h sqrt(tau_w,h)/nu (rho = 1); the
// enrichment function psi(y+) is Spalding's law (inverted by safeguarded Newton) or van Driest's
// law eq. (psi), evaluated as in Appendix A (Table A1 support points plus a 9-point Gauss rule,
// eq. psinum); grad psi = psi'(y+) grad y+ by the chain rule. The tables hold psi and grad psi at
// every quadrature point of the enriched cells and of their faces ("computed once ... and
// stored", Appendix A).
//
// Sec. 2.2: nu_t = l_mix^2 |eps(u~)| (eq. mix), l_mix = kappa y_DES (1 - exp(-y+/A+)) (eq. lmix),
// y_DES = (y^-beta + (C_DES h)^-beta)^(-1/beta) (eq. ydes) with h = dy_e/(k+1).
#include "metric.cuh"
#include "sumfac.cuh"

namespace dgw {

namespace {
constexpr double kKappa = 0.41;
constexpr double kAplus = 26.0;
constexpr double kBSpalding = 5.17;
constexpr double kCdes = 0.85;
constexpr double kBetaDes = 6.0;

__constant__ double c_vd_y[9] = {0.0, 5.0, 11.0, 24.0, 59.0, 144.0, 361.0, 946.0, 2517.0};
__constant__ double c_vd_psi[9] = {0.0, 4.88298776233176, 8.91824406645381, 12.3978516813118, 15.1875389926298,
                                   17.4177125619900, 19.6484300823042, 21.9930107788854, 24.3778307011372};
__constant__ double c_g9x[9];
__constant__ double c_g9w[9];
}  // namespace

__device__ double psi_spalding_dev(double yp, double *dpsi) {
  if (yp <= 0.0) { *dpsi = 1.0; return 0.0; }
  const double k = kKappa, eb = exp(-kKappa * kBSpalding);
  double lo = 0.0, hi = yp;
  double x = fmin(yp, kBSpalding + log1p(yp) / kKappa);
  for (int it = 0; it < 200; ++it) {
    const double kx = k * x;
    if (kx > 700.0) { hi = x; x = 0.5 * (lo + hi); continue; }
    const double e = exp(kx);
    const double g = x + eb * (e - 1.0 - kx - 0.5 * kx * kx - kx * kx * kx / 6.0) - yp;
    const double gp = 1.0 + eb * k * (e - 1.0 - kx - 0.5 * kx * kx);
    if (g > 0.0) hi = x; else lo = x;
    double xn = x - g / gp;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    const bool done = fabs(xn - x) <= 1e-16 * (1.0 + fabs(x));
    x = xn;
    if (done) break;
  }
  const double kx = k * x;
  *dpsi = 1.0 / (1.0 + eb * k * (exp(kx) - 1.0 - kx - 0.5 * kx * kx));
  return x;
}

__device__ __forceinline__ double vd_integrand(double y) {
  const double a = 2.0 * kKappa * y * (1.0 - exp(-y / kAplus));
  return 2.0 / (1.0 + sqrt(1.0 + a * a));
}

__device__ double psi_vandriest_dev(double yp, double *dpsi) {
  if (yp <= 0.0) { *dpsi = 1.0; return 0.0; }
  int i = 0;
  while (i < 8 && c_vd_y[i + 1] <= yp) ++i;
  const double a = c_vd_y[i], h = yp - a;
  double s = 0.0;
  for (int q = 0; q < 9; ++q) s += c_g9w[q] * vd_integrand(a + h * c_g9x[q]);
  *dpsi = vd_integrand(yp);
  return c_vd_psi[i] + h * s;
}

struct WallCellData {
  const double *ywall;   // [ne][8]
  const double *tauv;    // [ne][8]
  const int *enr_cell;   // [ne]
  MeshView<double> mv;   // geometry (boxes: row spacing; curved: metric tables)
  double nu;
  int wall_law;
};

// J^-1 at a point of cell c: boxes are diagonal; curved cells read the metric record (volume point
// (a0 of set sx, a1 of set sy), or face point (a1, a2) of face f with sets s1, s2 when f >= 0).
__device__ void point_metric(const WallCellData &w, const Basis<double> &B, int c, int f, int sx, int sy, int a0,
                             int a1, double Ji[3][3]) {
  const MeshView<double> &m = w.mv;
  if (m.geo == GEO_CURVED) {
    const int col = metric_col(m, c);
    const double *rec = f < 0 ? vol_rec(m, B, col, sx, sy, a0, a1) : face_rec(m, B, col, f >> 1, f & 1, sx, sy, a0, a1);
    double det;
    load_rec(rec, Ji, det);
    return;
  }
  const double h[3] = {m.hx, m.hy[(c / m.nx) % m.ny], m.hz};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Ji[a][b] = a == b ? 1.0 / h[a] : 0.0;
}

// Evaluate psi, grad psi, y_h and y+ at reference point xi of enriched cell e (J^-1 at the point).
__device__ void wall_point(const WallCellData &w, int e, const double xi[3], const double Ji[3][3], double out[WT],
                           double aux[2]) {
  double N[8], dN[8][3];
  q1_weights(xi, N, dN);
  double yh = 0.0, th = 0.0, gy[3] = {0, 0, 0}, gt[3] = {0, 0, 0};
  for (int v = 0; v < 8; ++v) {
    const double yv = w.ywall[8 * e + v], tv = w.tauv[8 * e + v];
    double g[3];
    ref_to_phys(Ji, dN[v], g);
    yh += N[v] * yv;
    th += N[v] * tv;
    for (int d = 0; d < 3; ++d) {
      gy[d] += g[d] * yv;
      gt[d] += g[d] * tv;
    }
  }
  const double st = sqrt(th);
  const double yp = yh * st / w.nu;
  double dpsi;
  const double psi = w.wall_law == 1 ? psi_vandriest_dev(yp, &dpsi) : psi_spalding_dev(yp, &dpsi);
  out[0] = psi;
  for (int d = 0; d < 3; ++d) out[1 + d] = dpsi * (st * gy[d] + yh * gt[d] / (2.0 * st)) / w.nu;
  aux[0] = yh;
  aux[1] = yp;
}

// Reference point of volume point t (x fastest; y uses the wall set) and of face point t, with the
// point's metric.
__device__ __forceinline__ void vol_xi(const WallCellData &w, const Basis<double> &B, int c, int qs, int t, double xi[3],
                                       double Ji[3][3]) {
  if (w.mv.full_q) qs = QSET_WALL;   // the q_w^3 rule
  const int q0 = B.q[qs], q1 = B.q[QSET_WALL];
  const int i0 = t % q0, i1 = (t / q0) % q1, i2 = t / (q0 * q1);
  xi[0] = B.x[qs][i0]; xi[1] = B.x[QSET_WALL][i1]; xi[2] = B.x[qs][i2];
  point_metric(w, B, c, -1, qs, QSET_WALL, i0, i1, Ji);
}
__device__ __forceinline__ bool face_xi(const WallCellData &w, const Basis<double> &B, int c, int qs, int f, int t,
                                        double xi[3], double Ji[3][3]) {
  const int d = f >> 1, side = f & 1;
  int t1, t2;
  face_axes(d, t1, t2);
  const int s1 = (t1 == 1 || w.mv.full_q) ? QSET_WALL : qs, s2 = (t2 == 1 || w.mv.full_q) ? QSET_WALL : qs;
  const int p1 = B.q[s1], p2 = B.q[s2];
  if (t >= p1 * p2) return false;
  xi[d] = side; xi[t1] = B.x[s1][t % p1]; xi[t2] = B.x[s2][t / p1];
  point_metric(w, B, c, f, s1, s2, t % p1, t / p1, Ji);
  return true;
}

// Squared mixing length l_mix^2 = (kappa y_DES (1 - exp(-y+/A+)))^2 (eq. lmix) with the smooth DES
// limiter y_DES = (y_h^-6 + (C_DES h)^-6)^(-1/6) (eq. ydes), h = wall-normal cell width / (k+1). It
// depends on the geometry and tau_w only, so it is tabulated with the wall tables and the eddy
// viscosity update multiplies it by the strain of the current field.
__device__ __forceinline__ double lmix_sq(double yh, double yp, double hdes) {
  double ydes = 0.0;
  if (yh > 0.0) ydes = pow(pow(yh, -kBetaDes) + pow(hdes, -kBetaDes), -1.0 / kBetaDes);
  const double lmix = kKappa * ydes * (1.0 - exp(-yp / kAplus));
  return lmix * lmix;
}

// aux records per linear-set point: (y_h, y+, l_mix^2)
constexpr int kAux = 3;

__global__ void wall_table_kernel(WallCellData w, const Basis<double> *Bg, int qs, int nvol, int fpmax,
                                  double *vol, double *face, double *aux_vol, double *aux_face, const double *dye,
                                  int k) {
  const Basis<double> &B = *Bg;
  const int e = blockIdx.x;
  const int c = w.enr_cell[e];
  const double hdes = dye ? kCdes * dye[e] / (k + 1) : 0.0;
  for (int t = threadIdx.x; t < nvol; t += blockDim.x) {
    double xi[3], Ji[3][3], out[WT], aux[2];
    vol_xi(w, B, c, qs, t, xi, Ji);
    wall_point(w, e, xi, Ji, out, aux);
    for (int r = 0; r < WT; ++r) vol[((size_t)e * nvol + t) * WT + r] = out[r];
    if (aux_vol) {
      double *a = aux_vol + ((size_t)e * nvol + t) * kAux;
      a[0] = aux[0]; a[1] = aux[1]; a[2] = lmix_sq(aux[0], aux[1], hdes);
    }
  }
  for (int t = threadIdx.x; t < 6 * fpmax; t += blockDim.x) {
    const int f = t / fpmax, pt = t % fpmax;
    double xi[3], Ji[3][3], out[WT] = {0, 0, 0, 0}, aux[2] = {0, 0};
    if (face_xi(w, B, c, qs, f, pt, xi, Ji)) wall_point(w, e, xi, Ji, out, aux);
    for (int r = 0; r < WT; ++r) face[((size_t)e * 6 * fpmax + t) * WT + r] = out[r];
    if (aux_face) {
      double *a = aux_face + ((size_t)e * 6 * fpmax + t) * kAux;
      a[0] = aux[0]; a[1] = aux[1]; a[2] = lmix_sq(aux[0], aux[1], hdes);
    }
  }
}

// nu_t at the linear-set volume and face points of enriched cell e from the enrichment
// coefficients of u.
__global__ void eddy_viscosity_kernel(WallCellData w, const Basis<double> *Bg, int nvol, int fpmax, const double *wt_vol,
                                      const double *wt_face, const double *aux_vol, const double *aux_face,
                                      const double *dye, int k, int nef, const double *u_enr, double *nut_vol, double *nut_face,
                                      float *nut_vol32, float *nut_face32) {
  const Basis<double> &B = *Bg;
  const int e = blockIdx.x;
  const int c = w.enr_cell[e];
  __shared__ double cu[24];
  for (int t = threadIdx.x; t < 24; t += blockDim.x) cu[t] = u_enr[(size_t)e * 3 * nef + (nef == 8 ? t : t >> 3)];
  __syncthreads();
  auto nut_at = [&](const double xi[3], const double Ji[3][3], const double *wt, const double *aux) -> double {
    // grad(psi sum_v N_v e_av) = psi J^-T (sum_v grad_xi N_v e_av) + (sum_v N_v e_av) grad psi, the sums
    // by nested linear interpolation
    const double f[3][2] = {{1.0 - xi[0], xi[0]}, {1.0 - xi[1], xi[1]}, {1.0 - xi[2], xi[2]}};
    double G[3][3];
    for (int a = 0; a < 3; ++a) {
      double sN, sD[3], gp[3];
      enr_trial<double, true>(f, cu + a * 8, nef == 1, sN, sD);
      ref_to_phys(Ji, sD, gp);
      for (int d = 0; d < 3; ++d) G[a][d] = wt[0] * gp[d] + sN * wt[1 + d];
    }
    double e2 = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) {
        const double eps = 0.5 * (G[a][d] + G[d][a]);
        e2 += eps * eps;
      }
    return aux[2] * sqrt(2.0 * e2);   // l_mix^2 |eps| (eq. mix), l_mix^2 tabulated per point
  };
  for (int t = threadIdx.x; t < nvol; t += blockDim.x) {
    double xi[3], Ji[3][3];
    vol_xi(w, B, c, QSET_LIN, t, xi, Ji);
    const size_t i = (size_t)e * nvol + t;
    const double v = nut_at(xi, Ji, wt_vol + i * WT, aux_vol + i * kAux);
    nut_vol[i] = v;
    if (nut_vol32) nut_vol32[i] = (float)v;
  }
  for (int t = threadIdx.x; t < 6 * fpmax; t += blockDim.x) {
    const int f = t / fpmax, pt = t % fpmax;
    double xi[3], Ji[3][3];
    const size_t i = (size_t)e * 6 * fpmax + t;
    double v = 0.0;
    if (face_xi(w, B, c, QSET_LIN, f, pt, xi, Ji)) v = nut_at(xi, Ji, wt_face + i * WT, aux_face + i * kAux);
    nut_face[i] = v;
    if (nut_face32) nut_face32[i] = (float)v;
  }
}

static WallCellData wall_data(dgw_mesh *M) {
  WallCellData w;
  w.ywall = M->wall_ywall_dev;
  w.tauv = M->wall_tauv_dev;
  w.enr_cell = M->enr_cell_dev;
  w.mv = M->v64;
  w.nu = M->P.nu;
  w.wall_law = M->P.wall_law;
  return w;
}

cudaError_t launch_wall_tables(dgw_mesh *M, cudaStream_t s) {
  if (M->ne == 0) return cudaSuccess;
  double gx[9], gw[9];
  gauss_rule(9, gx, gw);
  cudaError_t e = cudaMemcpyToSymbolAsync(c_g9x, gx, sizeof(gx), 0, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbolAsync(c_g9w, gw, sizeof(gw), 0, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  WallCellData w = wall_data(M);
  for (int cls = 0; cls < 2; ++cls) {
    const int qs = cls == 0 ? QSET_LIN : QSET_CONV;
    note_launch();
    wall_table_kernel<<<M->ne, 128, 0, s>>>(w, M->v64.basis, qs, M->v64.nvol[cls], M->v64.fpmax[cls],
                                            const_cast<double *>(M->v64.wt_vol[cls]),
                                            const_cast<double *>(M->v64.wt_face[cls]), cls == 0 ? M->aux_vol : nullptr,
                                            cls == 0 ? M->aux_face : nullptr, M->dye_dev, M->P.degree);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_eddy_viscosity(dgw_mesh *M, const double *u, cudaStream_t s) {
  if (M->ne == 0) return cudaSuccess;
  WallCellData w = wall_data(M);
  note_launch();
  eddy_viscosity_kernel<<<M->ne, 128, 0, s>>>(
      w, M->v64.basis, M->v64.nvol[0], M->v64.fpmax[0], M->v64.wt_vol[0], M->v64.wt_face[0], M->aux_vol, M->aux_face,
      M->dye_dev, M->P.degree, M->nef, u + 3 * M->np, const_cast<double *>(M->v64.nut_vol),
      const_cast<double *>(M->v64.nut_face), M->has32 ? const_cast<float *>(M->v32.nut_vol) : nullptr,
      M->has32 ? const_cast<float *>(M->v32.nut_face) : nullptr);
  return cudaGetLastError();
}

// Nodal wall shear stress (Sec. 3.2): tau_w,B = |int N_B nu (grad u_h) n dA| / int N_B dA over the
// wall faces, N_B the continuous bilinear functions of the wall vertices (periodic in x and z),
// k+1 Gauss points per tangential direction. One CTA per wall face (wall, i, k): every thread
// takes one face point and its traction; the 16 moments of the face (numerator and denominator of
// its four vertices) are summed over the points in a fixed order.
__global__ void wall_shear_face_kernel(MeshView<double> m, const double *__restrict__ u, const double *__restrict__ wt_face,
                                       int fpmax, double nu, double *__restrict__ out) {
  const Basis<double> &B = *m.basis;
  const int n = m.n1, n3 = n * n * n;
  const int b = blockIdx.x, wall = b / (m.nx * m.nz), r = b % (m.nx * m.nz), i = r % m.nx, kz = r / m.nx;
  const int j = wall ? m.ny - 1 : 0, c = i + m.nx * (j + m.ny * kz), side = wall;
  __shared__ double su[3 * NMAX * NMAX * NMAX], ce[24], mom[QMAX * QMAX][16];
  for (int t = threadIdx.x; t < 3 * n3; t += blockDim.x) su[t] = u[(size_t)c * 3 * n3 + t];
  const int e = m.enr ? m.enr[c] : -1;
  for (int t = threadIdx.x; t < 24; t += blockDim.x)
    ce[t] = e >= 0 ? u[3 * m.np + (size_t)e * 3 * m.nef + (m.nef == 8 ? t : t >> 3)] : 0.0;
  __syncthreads();
  // k+1 points per direction; q_w on the wall faces of enriched cells under the q_w^3 rule
  const int sq = (m.full_q && e >= 0) ? QSET_WALL : QSET_LIN, pq = B.q[sq], npts = pq * pq;
  const double *S = B.S[sq], *D = B.D[sq], *de = B.dend[side];
  const int jend = side ? n - 1 : 0;
  for (int t = threadIdx.x; t < npts; t += blockDim.x) {
    const int a1 = t % pq, a2 = t / pq;
    const double xi[3] = {B.x[sq][a1], (double)side, B.x[sq][a2]};
    double Ji[3][3], det;
    if (m.geo == GEO_CURVED) {
      load_rec(face_rec(m, B, metric_col(m, c), 1, side, sq, sq, a1, a2), Ji, det);
    } else {
      const double h[3] = {m.hx, m.hy[j], m.hz};
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) Ji[p][q] = p == q ? 1.0 / h[p] : 0.0;
      det = h[0] * h[1] * h[2];
    }
    // reference gradient of the standard part (Gauss-Lobatto nodes: the face layer is node row jend)
    double G[3][3];
    for (int a = 0; a < 3; ++a) {
      const double *ua = su + a * n3;
      double g[3] = {0.0, 0.0, 0.0};
      for (int l = 0; l < n; ++l)
        for (int ii = 0; ii < n; ++ii) {
          const double ul = ua[ii + n * (jend + n * l)];
          g[0] += D[a1 * n + ii] * S[a2 * n + l] * ul;
          g[2] += S[a1 * n + ii] * D[a2 * n + l] * ul;
          double s1 = 0.0;
          for (int jj = 0; jj < n; ++jj) s1 += de[jj] * ua[ii + n * (jj + n * l)];
          g[1] += S[a1 * n + ii] * S[a2 * n + l] * s1;
        }
      ref_to_phys(Ji, g, G[a]);
    }
    // enrichment: grad(psi N_v) = psi grad N_v + N_v grad psi, psi and grad psi from the wall table
    if (e >= 0) {
      const double *wt = wt_face + (((size_t)e * 6 + 2 + side) * fpmax + t) * WT;
      const double f[3][2] = {{1.0 - xi[0], xi[0]}, {1.0 - xi[1], xi[1]}, {1.0 - xi[2], xi[2]}};
      for (int a = 0; a < 3; ++a) {
        double sN, sD[3], gp[3];
        enr_trial<double, true>(f, ce + a * 8, m.nef == 1, sN, sD);
        ref_to_phys(Ji, sD, gp);
        for (int d = 0; d < 3; ++d) G[a][d] += wt[0] * gp[d] + sN * wt[1 + d];
      }
    }
    // outward unit normal and area weight of the face xi_1 = side (Nanson)
    const double gl = sqrt(Ji[1][0] * Ji[1][0] + Ji[1][1] * Ji[1][1] + Ji[1][2] * Ji[1][2]);
    const double sg = side ? 1.0 : -1.0;
    const double nrm[3] = {sg * Ji[1][0] / gl, sg * Ji[1][1] / gl, sg * Ji[1][2] / gl};
    const double dA = fabs(det) * gl * B.w[sq][a1] * B.w[sq][a2];
    double tw[3];
    for (int a = 0; a < 3; ++a) tw[a] = nu * (G[a][0] * nrm[0] + G[a][1] * nrm[1] + G[a][2] * nrm[2]);
    for (int v = 0; v < 4; ++v) {
      const double Nb = ((v & 1) ? xi[0] : 1.0 - xi[0]) * ((v & 2) ? xi[2] : 1.0 - xi[2]);
      for (int a = 0; a < 3; ++a) mom[t][v * 4 + a] = Nb * tw[a] * dA;
      mom[t][v * 4 + 3] = Nb * dA;
    }
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    double acc = 0.0;
    for (int t = 0; t < npts; ++t) acc += mom[t][threadIdx.x];
    out[(size_t)b * 16 + threadIdx.x] = acc;
  }
}

// tau_w,B per wall node from the moments of its (up to) four faces, in a fixed order
__global__ void wall_shear_node_kernel(const double *__restrict__ mom, int nx, int nz, double *__restrict__ tau) {
  const int nn = 2 * nx * nz;
  for (int bnode = blockIdx.x * blockDim.x + threadIdx.x; bnode < nn; bnode += gridDim.x * blockDim.x) {
    const int wall = bnode / (nx * nz), r = bnode % (nx * nz), i = r % nx, k = r / nx;
    double num[3] = {0.0, 0.0, 0.0}, den = 0.0;
    for (int dk = 0; dk < 2; ++dk)
      for (int da = 0; da < 2; ++da) {
        const int fi = (i - da + nx) % nx, fk = (k - dk + nz) % nz;
        const double *f = mom + ((size_t)wall * nx * nz + fi + nx * fk) * 16 + (da + 2 * dk) * 4;
        for (int a = 0; a < 3; ++a) num[a] += f[a];
        den += f[3];
      }
    tau[bnode] = sqrt(num[0] * num[0] + num[1] * num[1] + num[2] * num[2]) / den;
  }
}

// vertex values of the enriched cells from the wall nodes that define their wall distances
__global__ void tau_fill_kernel(const double *__restrict__ tau_nodes, const int *__restrict__ tsrc, int n,
                                double *__restrict__ tauv) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) tauv[i] = tau_nodes[tsrc[i]];
}

cudaError_t launch_wall_shear(dgw_mesh *M, const double *u, double *tau_nodes, cudaStream_t s) {
  const int nf = 2 * M->P.nx * M->P.nz;
  note_launches(2);
  wall_shear_face_kernel<<<nf, 64, 0, s>>>(M->v64, u, M->v64.wt_face[0], M->v64.fpmax[0], M->P.nu, M->wall_mom_dev);
  wall_shear_node_kernel<<<(nf + 255) / 256, 256, 0, s>>>(M->wall_mom_dev, M->P.nx, M->P.nz, tau_nodes);
  return cudaGetLastError();
}

// Switch-off of the wall model (Sec. 3.2): enriched cell e is on iff some point of the velocity point
// set of the wall-nearest cell of its column has y+ >= yp_off (aux_vol holds (y_h, y+, l_mix^2) per point of
// every enriched cell, switched on or not). Writes the operators' view enr[c].
__global__ void switch_kernel(const double *__restrict__ aux_vol, int nvol, const int *__restrict__ wslot,
                              const int *__restrict__ enr_cell, int ne, double yp_off, int *__restrict__ enr) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
    const double *a = aux_vol + (size_t)wslot[e] * nvol * kAux;
    double ymax = 0.0;
    for (int t = 0; t < nvol; ++t) ymax = fmax(ymax, a[kAux * t + 1]);
    enr[enr_cell[e]] = ymax < yp_off ? -1 : e;
  }
}

cudaError_t launch_switch(dgw_mesh *M, cudaStream_t s) {
  M->mass_factor_valid = false;   // the cell spaces may change
  if (M->ne == 0) return cudaSuccess;
  note_launch();
  switch_kernel<<<(M->ne + 127) / 128, 128, 0, s>>>(M->aux_vol, M->v64.nvol[0], M->wslot_dev, M->enr_cell_dev, M->ne,
                                                    M->yp_off, const_cast<int *>(M->v64.enr));
  return cudaGetLastError();
}

cudaError_t launch_set_tau_nodes(dgw_mesh *M, const double *tau_nodes, cudaStream_t s) {
  if (M->ne == 0) return cudaSuccess;
  note_launch();
  tau_fill_kernel<<<(8 * M->ne + 255) / 256, 256, 0, s>>>(tau_nodes, M->tsrc_dev, 8 * M->ne, M->wall_tauv_dev);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_wall_tables(M, s);
  if (e == cudaSuccess) e = launch_switch(M, s);
  if (e == cudaSuccess && M->has32)
    for (int cls = 0; cls < 2 && e == cudaSuccess; ++cls) {
      e = launch_to_float(M->v64.wt_vol[cls], const_cast<float *>(M->v32.wt_vol[cls]),
                          (size_t)M->ne * M->v64.nvol[cls] * WT, s);
      if (e == cudaSuccess)
        e = launch_to_float(M->v64.wt_face[cls], const_cast<float *>(M->v32.wt_face[cls]),
                            (size_t)M->ne * 6 * M->v64.fpmax[cls] * WT, s);
    }
  return e;
}

// float copies of the wall tables
__global__ void to_float_kernel(const double *a, float *b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

cudaError_t launch_to_float(const double *a, float *b, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  note_launch();
  to_float_kernel<<<1216, 256, 0, s>>>(a, b, n);
  return cudaGetLastError();
}

}  // namespace dgw
