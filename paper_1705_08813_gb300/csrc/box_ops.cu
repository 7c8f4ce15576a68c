// Degree-specialised DG operators on the box cells of the channel whose six neighbours are
// standard cells (Sec. 4.2 weak forms, Sec. 4.4 sum factorisation); the enriched wall layers and
// the rows next to them take the general kernel of ops.cu.
//
// On an axis-aligned box every integrand of the divergence and of the viscous term is a
// polynomial of degree <= 2k per direction, which the k+1 Gauss points of these terms integrate
// exactly. Their volume integrals are therefore Kronecker products of 1-D matrices over the
// Gauss-Lobatto nodes, M_ij = (l_i, l_j), K_ij = (l_i', l_j'), A_ij = (l_i', l_j) (test
// derivative, trial value) and B = A^T, with no interpolation to points; on the faces the traces
// are the nodal values of the face layer (the end nodes of the Lobatto lines), normal derivatives
// come from the end-point derivatives l_j'(0), l_j'(1), tangential ones from the nodal
// differentiation matrix, and the face integrals are (M x M)-type products on the n x n face grid.
// The result equals the Gauss-point evaluation up to rounding.
//
// Every kernel is templated on the storage type T of the vectors and the compute type R (T itself,
// or df64 for FP64-accurate double-float arithmetic on the FP32 units with double vectors). A CTA
// holds cpb consecutive cells of one row segment along x; each thread owns one line of one cell in
// every pass (x-, y- then z-lines) and, in the face phase of direction d, the d-line through its
// face node.
#include <cmath>
#include <cstring>
#include <mutex>
#include <utility>
#include <type_traits>

#include "df64.cuh"
#include "metric.cuh"
#include "sumfac.cuh"

namespace dgw {

// 1-D tables of one degree on the Gauss-Lobatto nodes; Sc, Dc, wc: the convective point set
// (floor(3k/2)+1 Gauss points), rows = points.
template <typename R>
struct VecConst {
  R M[NMAX * NMAX];
  R K[NMAX * NMAX];
  R A[NMAX * NMAX];
  R Dg[NMAX * NMAX];   // Dg[i * n + j] = l_j'(x_i) at the Lobatto nodes
  R de[2][NMAX];       // l_j'(0), l_j'(1)
  R Sc[QMAX * NMAX];
  R Dc[QMAX * NMAX];
  R wc[QMAX];
  // Even-odd halves of Sc and Dc (the point set and the nodes are symmetric about 1/2, so
  // Sc[q-1-j][n-1-b] = Sc[j][b] and Dc[q-1-j][n-1-b] = -Dc[j][b]), rows j < q/2, columns b < n/2,
  // stride n: SE/SO = (Sc[j][b] +/- Sc[j][n-1-b]) / 2, DA/DB = (Dc[j][b] -/+ Dc[j][n-1-b]) / 2
  R SE[(QMAX / 2) * NMAX];
  R SO[(QMAX / 2) * NMAX];
  R DA[(QMAX / 2) * NMAX];
  R DB[(QMAX / 2) * NMAX];
  // the enriched neighbour's trace on a y-face: positions of the k+1 Gauss points (xg) and of the
  // convective points (xc) on [0, 1], and Sinv[b * n + t], the inverse of the k+1-point value table
  // (nodal values whose interpolant takes given values at the Gauss points)
  R xg[NMAX];
  R xc[QMAX];
  R Sinv[NMAX * NMAX];
  // even-odd halves of the n x n node matrices, rows r < n/2, columns b < n/2, stride n:
  // X_E/X_O = (X[r][b] +/- X[r][n-1-b]) / 2 for X = M, K (centro-symmetric), A and A^T
  // (centro-antisymmetric: X[n-1-r][n-1-b] = -X[r][b])
  R ME[(NMAX / 2) * NMAX], MO[(NMAX / 2) * NMAX];
  R KE[(NMAX / 2) * NMAX], KO[(NMAX / 2) * NMAX];
  R AE[(NMAX / 2) * NMAX], AO[(NMAX / 2) * NMAX];
  R TE[(NMAX / 2) * NMAX], TO[(NMAX / 2) * NMAX];
};
// the three tables share the 64 KB constant bank of this translation unit
static_assert(5 * (2 * sizeof(VecConst<double>) + sizeof(VecConst<float>)) <= 62 * 1024, "constant tables too large");
__constant__ VecConst<double> c_vec64[5];
__constant__ VecConst<float> c_vec32[5];
__constant__ VecConst<df64> c_vecdf[5];

template <typename R>
__device__ __forceinline__ const VecConst<R> &vconst(int k);
template <>
__device__ __forceinline__ const VecConst<double> &vconst<double>(int k) { return c_vec64[k - 1]; }
template <>
__device__ __forceinline__ const VecConst<float> &vconst<float>(int k) { return c_vec32[k - 1]; }
template <>
__device__ __forceinline__ const VecConst<df64> &vconst<df64>(int k) { return c_vecdf[k - 1]; }

template <typename R>
__device__ __forceinline__ R r_from_double(double x);
template <>
__device__ __forceinline__ double r_from_double<double>(double x) { return x; }
template <>
__device__ __forceinline__ float r_from_double<float>(double x) { return (float)x; }
template <>
__device__ __forceinline__ df64 r_from_double<df64>(double x) { return df_from(x); }

// out = Mat in along a line (Mat n x n row-major, or its transpose)
template <typename R, int n, bool TR = false>
__device__ __forceinline__ void matvec(const R *Mat, const R (&in)[n], R (&out)[n]) {
#pragma unroll
  for (int r = 0; r < n; ++r) {
    R s = r_zero<R>();
#pragma unroll
    for (int b = 0; b < n; ++b) s = r_fma(TR ? Mat[b * n + r] : Mat[r * n + b], in[b], s);
    out[r] = s;
  }
}
// Even-odd form of out (=|+= c *) X in for an n x n node matrix X with X[n-1-r][n-1-b] = SIG X[r][b]
// (E, O its halves, F the full matrix, read transposed when TR, for the middle row and column):
// out[r] = e_r + o_r and out[n-1-r] = SIG (e_r - o_r) from products with the sums and differences of
// mirrored inputs; the middle row (odd n) takes the sums (SIG = 1) or the differences (SIG = -1).
template <typename R, int n, int SIG, bool TR, bool ACC>
__device__ __forceinline__ void matvec_eo(const R *E, const R *O, const R *F, R c, const R (&v)[n], R (&out)[n]) {
  constexpr int nh = n / 2;
  R ve[nh > 0 ? nh : 1], vo[nh > 0 ? nh : 1];
#pragma unroll
  for (int b = 0; b < nh; ++b) { ve[b] = v[b] + v[n - 1 - b]; vo[b] = v[b] - v[n - 1 - b]; }
#pragma unroll
  for (int r = 0; r < nh; ++r) {
    R e = (n & 1) ? (TR ? F[nh * n + r] : F[r * n + nh]) * v[nh] : r_zero<R>(), o = r_zero<R>();
#pragma unroll
    for (int b = 0; b < nh; ++b) {
      e = r_fma(E[r * n + b], ve[b], e);
      o = r_fma(O[r * n + b], vo[b], o);
    }
    const R lo = e + o, hi = SIG > 0 ? e - o : o - e;
    out[r] = ACC ? r_fma(c, lo, out[r]) : lo;
    out[n - 1 - r] = ACC ? r_fma(c, hi, out[n - 1 - r]) : hi;
  }
  if constexpr ((n & 1) != 0) {
    R m = SIG > 0 ? F[nh * n + nh] * v[nh] : r_zero<R>();
#pragma unroll
    for (int b = 0; b < nh; ++b) m = r_fma(TR ? F[b * n + nh] : F[nh * n + b], SIG > 0 ? ve[b] : vo[b], m);
    out[nh] = ACC ? r_fma(c, m, out[nh]) : m;
  }
}
template <typename R, int n>
__device__ __forceinline__ void mv_M(const VecConst<R> &C, const R (&v)[n], R (&o)[n]) {
  matvec_eo<R, n, 1, false, false>(C.ME, C.MO, C.M, r_zero<R>(), v, o);
}
template <typename R, int n>
__device__ __forceinline__ void mv_K(const VecConst<R> &C, const R (&v)[n], R (&o)[n]) {
  matvec_eo<R, n, 1, false, false>(C.KE, C.KO, C.K, r_zero<R>(), v, o);
}
template <typename R, int n>
__device__ __forceinline__ void mv_A(const VecConst<R> &C, const R (&v)[n], R (&o)[n]) {
  matvec_eo<R, n, -1, false, false>(C.AE, C.AO, C.A, r_zero<R>(), v, o);
}
template <typename R, int n>
__device__ __forceinline__ void mv_AT(const VecConst<R> &C, const R (&v)[n], R (&o)[n]) {
  matvec_eo<R, n, -1, true, false>(C.TE, C.TO, C.A, r_zero<R>(), v, o);
}
template <typename R, int n>
__device__ __forceinline__ void mva_M(const VecConst<R> &C, R c, const R (&v)[n], R (&o)[n]) {
  matvec_eo<R, n, 1, false, true>(C.ME, C.MO, C.M, c, v, o);
}
template <typename R, int n>
__device__ __forceinline__ void mva_K(const VecConst<R> &C, R c, const R (&v)[n], R (&o)[n]) {
  matvec_eo<R, n, 1, false, true>(C.KE, C.KO, C.K, c, v, o);
}
template <typename R, int n>
__device__ __forceinline__ void mva_A(const VecConst<R> &C, R c, const R (&v)[n], R (&o)[n]) {
  matvec_eo<R, n, -1, false, true>(C.AE, C.AO, C.A, c, v, o);
}

// out += c * Mat in
template <typename R, int n, bool TR = false>
__device__ __forceinline__ void matvec_acc(const R *Mat, R c, const R (&in)[n], R (&out)[n]) {
#pragma unroll
  for (int r = 0; r < n; ++r) {
    R s = r_zero<R>();
#pragma unroll
    for (int b = 0; b < n; ++b) s = r_fma(TR ? Mat[b * n + r] : Mat[r * n + b], in[b], s);
    out[r] = r_fma(c, s, out[r]);
  }
}

template <typename R, int n>
__device__ __forceinline__ void load_line(const R *p, int stride, R (&v)[n]) {
#pragma unroll
  for (int b = 0; b < n; ++b) v[b] = p[b * stride];
}
template <typename R, int n>
__device__ __forceinline__ void store_line(R *p, int stride, const R (&v)[n]) {
#pragma unroll
  for (int b = 0; b < n; ++b) p[b * stride] = v[b];
}

// Even-odd forms of the 1-D products with the convective point set (Kronbichler and Kormann's even-odd
// decomposition for symmetric 1-D bases): with v_e/v_o the sums and differences of mirrored entries,
// each pair of mirrored outputs takes one product with a half-size table, about 4/5 of the
// multiply-adds of the plain product at n = 5, q = 7.
// out = Sc v (q points from n nodes)
template <typename R, int n, int q>
__device__ __forceinline__ void interp_eo(const VecConst<R> &C, const R (&v)[n], R (&out)[q]) {
  constexpr int nh = n / 2, qh = q / 2;
  R ve[nh > 0 ? nh : 1], vo[nh > 0 ? nh : 1];
#pragma unroll
  for (int b = 0; b < nh; ++b) { ve[b] = v[b] + v[n - 1 - b]; vo[b] = v[b] - v[n - 1 - b]; }
#pragma unroll
  for (int i = 0; i < qh; ++i) {
    R e = (n & 1) ? C.Sc[i * n + nh] * v[nh] : r_zero<R>(), o = r_zero<R>();
#pragma unroll
    for (int b = 0; b < nh; ++b) {
      e = r_fma(C.SE[i * n + b], ve[b], e);
      o = r_fma(C.SO[i * n + b], vo[b], o);
    }
    out[i] = e + o;
    out[q - 1 - i] = e - o;
  }
  if constexpr ((q & 1) != 0) {
    R m = (n & 1) ? C.Sc[qh * n + nh] * v[nh] : r_zero<R>();
#pragma unroll
    for (int b = 0; b < nh; ++b) m = r_fma(C.Sc[qh * n + b], ve[b], m);
    out[qh] = m;
  }
}
// sums and differences of mirrored point values
template <typename R, int q>
__device__ __forceinline__ void point_eo(const R (&f)[q], R (&fe)[q / 2 > 0 ? q / 2 : 1], R (&fo)[q / 2 > 0 ? q / 2 : 1]) {
#pragma unroll
  for (int j = 0; j < q / 2; ++j) { fe[j] = f[j] + f[q - 1 - j]; fo[j] = f[j] - f[q - 1 - j]; }
}
// out (+)= Sc^T f (n nodes from q points; fe/fo from point_eo, fm = f[q/2] when q is odd)
template <typename R, int n, int q, bool ACC>
__device__ __forceinline__ void tinterp_s_eo(const VecConst<R> &C, const R (&fe)[q / 2 > 0 ? q / 2 : 1],
                                             const R (&fo)[q / 2 > 0 ? q / 2 : 1], R fm, R (&out)[n]) {
  constexpr int nh = n / 2, qh = q / 2;
#pragma unroll
  for (int b = 0; b < nh; ++b) {
    R e = (q & 1) ? C.Sc[qh * n + b] * fm : r_zero<R>(), o = r_zero<R>();
#pragma unroll
    for (int j = 0; j < qh; ++j) {
      e = r_fma(C.SE[j * n + b], fe[j], e);
      o = r_fma(C.SO[j * n + b], fo[j], o);
    }
    out[b] = ACC ? out[b] + (e + o) : e + o;
    out[n - 1 - b] = ACC ? out[n - 1 - b] + (e - o) : e - o;
  }
  if constexpr ((n & 1) != 0) {
    R m = (q & 1) ? C.Sc[qh * n + nh] * fm : r_zero<R>();
#pragma unroll
    for (int j = 0; j < qh; ++j) m = r_fma(C.Sc[j * n + nh], fe[j], m);
    out[nh] = ACC ? out[nh] + m : m;
  }
}
// out (+)= Dc^T f
template <typename R, int n, int q, bool ACC>
__device__ __forceinline__ void tinterp_d_eo(const VecConst<R> &C, const R (&fe)[q / 2 > 0 ? q / 2 : 1],
                                             const R (&fo)[q / 2 > 0 ? q / 2 : 1], R fm, R (&out)[n]) {
  constexpr int nh = n / 2, qh = q / 2;
#pragma unroll
  for (int b = 0; b < nh; ++b) {
    R e = (q & 1) ? C.Dc[qh * n + b] * fm : r_zero<R>(), o = r_zero<R>();
#pragma unroll
    for (int j = 0; j < qh; ++j) {
      e = r_fma(C.DA[j * n + b], fe[j], e);
      o = r_fma(C.DB[j * n + b], fo[j], o);
    }
    out[b] = ACC ? out[b] + (e + o) : e + o;
    out[n - 1 - b] = ACC ? out[n - 1 - b] + (o - e) : o - e;
  }
  if constexpr ((n & 1) != 0) {
    R m = r_zero<R>();   // the middle node's derivative is odd about the middle point
#pragma unroll
    for (int j = 0; j < qh; ++j) m = r_fma(C.Dc[j * n + nh], fo[j], m);
    out[nh] = ACC ? out[nh] + m : m;
  }
}

// Enrichment of a neighbour across a y-face, as seen from a standard cell of the rows next to the
// enriched layers (Sec. 3, u~ = psi sum_B N_B u~_B on the neighbour). On the face the neighbour sits
// at xi_y = 1 - s (s: the own face side), so only its four trilinear weights of that layer are
// nonzero there, bilinear in the tangential positions x, z; with l = 0 the sum is the single
// coefficient. e4 holds those four coefficients (x fastest), or the single one in e4[0].
template <typename T, typename R>
__device__ __forceinline__ void enr_face_coeffs(const MeshView<T> &m, const T *__restrict__ u, int eb, int s, int a,
                                                R (&e4)[4]) {
  const T *e = u + 3 * m.np + ((size_t)eb * 3 + a) * m.nef;
  if (m.nef == 1) {
    e4[0] = e4[1] = e4[2] = e4[3] = r_load<R>(e[0]);
    return;
  }
  const int by = 2 * (1 - s);
  e4[0] = r_load<R>(e[by]);
  e4[1] = r_load<R>(e[by + 1]);
  e4[2] = r_load<R>(e[by + 4]);
  e4[3] = r_load<R>(e[by + 5]);
}
template <typename R>
__device__ __forceinline__ R enr_face_sum(const R (&e4)[4], bool l0, R x, R z) {
  if (l0) return e4[0];
  const R one = r_from_double<R>(1.0);
  const R x0 = one - x, z0 = one - z;
  return r_fma(x * z, e4[3], r_fma(x0 * z, e4[2], r_fma(x * z0, e4[1], (x0 * z0) * e4[0])));
}
// Nodal values g at face node (i1, i2) (t1 = x, t2 = z) of components a0 .. a0 + NA - 1 whose
// interpolant takes the neighbour eb's enrichment psi sum_v N_v e_av at the k+1 Gauss points of the
// face (psi from the neighbour's wall table of that face). The node-space face integrals use
// M = S^T W S, so integrating g reproduces the Gauss-point integral of the enrichment exactly.
template <typename T, typename R, int n, int NA>
__device__ __forceinline__ void enr_face_nodal(const VecConst<R> &C, const MeshView<T> &m, const T *__restrict__ u,
                                               int eb, int s, int a0, int i1, int i2, R (&g)[NA]) {
  const T *w = m.wt_face[0] + ((size_t)eb * 6 + 2 + (1 - s)) * m.fpmax[0] * WT;
  const bool l0 = m.nef == 1;
  R e4[NA][4];
#pragma unroll
  for (int c = 0; c < NA; ++c) {
    enr_face_coeffs<T, R>(m, u, eb, s, a0 + c, e4[c]);
    g[c] = r_zero<R>();
  }
#pragma unroll 1
  for (int j2 = 0; j2 < n; ++j2) {
    R row[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) row[c] = r_zero<R>();
#pragma unroll
    for (int j1 = 0; j1 < n; ++j1) {
      const R sp = C.Sinv[i1 * n + j1] * r_load<R>(w[(j1 + n * j2) * WT]);
#pragma unroll
      for (int c = 0; c < NA; ++c) row[c] = r_fma(sp, enr_face_sum<R>(e4[c], l0, C.xg[j1], C.xg[j2]), row[c]);
    }
#pragma unroll
    for (int c = 0; c < NA; ++c) g[c] = r_fma(C.Sinv[i2 * n + j2], row[c], g[c]);
  }
}

// line of a pass: x-lines (base n l, stride 1), y-lines (base lr + n^2 lq, stride n), z-lines
// (base l, stride n^2)
template <int n>
__device__ __forceinline__ void line_geom(int d, int l, int &base, int &stride) {
  const int lr = l % n, lq = l / n;
  if (d == 0) { base = n * l; stride = 1; }
  else if (d == 1) { base = lr + n * n * lq; stride = n; }
  else { base = l; stride = n * n; }
}

// Cells of one CTA: cpb consecutive cells of row j0 + (blockIdx / segments) % nrows, plane kz.
struct BoxBlock {
  int c0, i0, j, kz;
};
template <typename T>
__device__ __forceinline__ BoxBlock box_block(const MeshView<T> &m, int cpb, int j0, int nrows) {
  const int segs = m.nx / cpb;
  const int b = blockIdx.x;
  BoxBlock r;
  r.i0 = (b % segs) * cpb;
  r.j = j0 + (b / segs) % nrows;
  r.kz = b / (segs * nrows);
  r.c0 = r.i0 + m.nx * (r.j + m.ny * r.kz);
  return r;
}

// The d-line of the neighbour across face (d, s) of cell c (component a, ncomp components per
// cell): from shared memory when the neighbour is one of the CTA's cells, else from global memory.
template <typename T, typename R, int n>
__device__ __forceinline__ void neighbour_line(const R *U, const T *__restrict__ u, int nb, const BoxBlock &bk, int cpb,
                                               int ncomp, int a, int base, int stride, R (&v)[n]) {
  constexpr int n3 = n * n * n;
  const int rel = nb - bk.c0;
  if (rel >= 0 && rel < cpb) {
    load_line<R, n>(U + (rel * ncomp + a) * n3 + base, stride, v);
  } else {
    const T *p = u + ((size_t)nb * ncomp + a) * n3 + base;
#pragma unroll
    for (int b = 0; b < n; ++b) v[b] = r_load<R>(p[b * stride]);
  }
}

// ------------------------------------------------------------------------------------------------
// Divergence b = -C(q, u) (Sec. 4.2): sum_d (d q / d x_d, u_d)_K - (q, {{u}}.n)_dK with {{u}} = u^-
// on walls. Volume: V sum_d (1/h_d) (A_d x M x M) u_d. Faces (normal d, side s, sgn = 2s - 1):
// -|F| sgn (M x M) {{u_d}} on the face layer.
// ------------------------------------------------------------------------------------------------
template <typename T, typename R, int K>
__global__ void __launch_bounds__(128) box_div_kernel(MeshView<T> m, const T *__restrict__ u, T *__restrict__ y, int cpb,
                                                      int j0, int nrows) {
  constexpr int n = K + 1, n2 = n * n, n3 = n2 * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *U = reinterpret_cast<R *>(smem_raw);   // cpb x 3 x n3
  R *Y = U + cpb * 3 * n3;                   // cpb x n3
  R *S = Y + cpb * n3;                       // cpb x 3 x n3 scratch
  const VecConst<R> &C = vconst<R>(K);
  const int tid = threadIdx.x, nt = blockDim.x;
  const BoxBlock bk = box_block(m, cpb, j0, nrows);
  for (int t = tid; t < cpb * 3 * n3; t += nt) U[t] = r_load<R>(u[(size_t)bk.c0 * 3 * n3 + t]);
  const double hd[3] = {(double)m.hx, (double)m.hy[bk.j], (double)m.hz};
  const double V = hd[0] * hd[1] * hd[2];
  const R sx = r_from_double<R>(V / hd[0]), sy = r_from_double<R>(V / hd[1]), sz = r_from_double<R>(V / hd[2]);
  __syncthreads();
  const bool line = tid < cpb * n2;
  const int cl = line ? tid / n2 : 0, l = line ? tid - cl * n2 : 0;
  R *Uc = U + cl * 3 * n3, *Yc = Y + cl * n3, *Sc = S + cl * 3 * n3;
  // x-lines: P0 = A_x u0, P1 = M_x u1, P2 = M_x u2
  if (line) {
    int base, st;
    line_geom<n>(0, l, base, st);
    R v[n], o[n];
    load_line<R, n>(Uc + base, st, v);
    mv_A<R, n>(C, v, o);
    store_line<R, n>(Sc + base, st, o);
    load_line<R, n>(Uc + n3 + base, st, v);
    mv_M<R, n>(C, v, o);
    store_line<R, n>(Sc + n3 + base, st, o);
    load_line<R, n>(Uc + 2 * n3 + base, st, v);
    mv_M<R, n>(C, v, o);
    store_line<R, n>(Sc + 2 * n3 + base, st, o);
  }
  __syncthreads();
  // y-lines: W = sx M_y P0 + sy A_y P1, T = M_y P2
  if (line) {
    int base, st;
    line_geom<n>(1, l, base, st);
    R p0[n], p1[n], p2[n], w[n], t[n];
    load_line<R, n>(Sc + base, st, p0);
    load_line<R, n>(Sc + n3 + base, st, p1);
    load_line<R, n>(Sc + 2 * n3 + base, st, p2);
#pragma unroll
    for (int r = 0; r < n; ++r) w[r] = r_zero<R>();
    mva_M<R, n>(C, sx, p0, w);
    mva_A<R, n>(C, sy, p1, w);
    mv_M<R, n>(C, p2, t);
    store_line<R, n>(Sc + base, st, w);
    store_line<R, n>(Sc + n3 + base, st, t);
  }
  __syncthreads();
  // z-lines: y = M_z W + sz A_z T
  if (line) {
    int base, st;
    line_geom<n>(2, l, base, st);
    R w[n], t[n], o[n];
    load_line<R, n>(Sc + base, st, w);
    load_line<R, n>(Sc + n3 + base, st, t);
    mv_M<R, n>(C, w, o);
    mva_A<R, n>(C, sz, t, o);
    store_line<R, n>(Yc + base, st, o);
  }
  __syncthreads();
  // faces: -|F| sgn (M x M) {{u_d}} on the layer of each face
  R *F = S + cl * 4 * n2;   // [face s][stage][n2] (the volume scratch is free now)
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int t1, t2;
    face_axes(d, t1, t2);
    const R area = r_from_double<R>(-V / hd[d]);
    const int i1 = l % n, i2 = l / n;
    int base, st;
    line_geom<n>(d, l, base, st);
    if (line) {
      for (int s = 0; s < 2; ++s) {
        const int c = bk.c0 + cl;
        const int nb = neighbour(m, c, 2 * d + s);
        const R own = Uc[d * n3 + base + (s ? n - 1 : 0) * st];
        R avg = own;
        if (nb >= 0) {
          R v[n];
          neighbour_line<T, R, n>(U, u, nb, bk, cpb, 3, d, base, st, v);
          R other = v[s ? 0 : n - 1];
          const int eb = d == 1 ? m.enr[nb] : -1;
          if (eb >= 0) {   // the enriched neighbour's u~_y on the face
            R g[1];
            enr_face_nodal<T, R, n, 1>(C, m, u, eb, s, 1, i1, i2, g);
            other = other + g[0];
          }
          avg = r_half<R>() * (own + other);
        }
        F[s * 2 * n2 + l] = (s ? area : -area) * avg;   // sgn(s) * (-|F|) * avg
      }
    }
    __syncthreads();
    if (line) {   // along t1
      for (int s = 0; s < 2; ++s) {
        R acc = r_zero<R>();
#pragma unroll
        for (int r = 0; r < n; ++r) acc = r_fma(C.M[i1 * n + r], F[s * 2 * n2 + r + n * i2], acc);
        F[s * 2 * n2 + n2 + l] = acc;
      }
    }
    __syncthreads();
    if (line) {   // along t2, add to the layer
      for (int s = 0; s < 2; ++s) {
        R acc = r_zero<R>();
#pragma unroll
        for (int r = 0; r < n; ++r) acc = r_fma(C.M[i2 * n + r], F[s * 2 * n2 + n2 + i1 + n * r], acc);
        Yc[base + (s ? n - 1 : 0) * st] += acc;
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < cpb * n3; t += nt) y[(size_t)bk.c0 * n3 + t] = r_store<T>(Y[t]);
}

// ------------------------------------------------------------------------------------------------
// Viscous term -F^nu(v, u) of standard cells (eq. viscous_multiscale with no enrichment on either
// side of any face): (eps(v), 2 nu eps(u))_K + on each face (1/2 F^nu(v), [[u]]) - (v, {{F^nu(u)}}.n)
// + (v, tau_F nu [[u]].n), tau_F = max of the two cells, 10 tau on walls, mirror state on walls.
// Volume for output a: nu V [ sum_d (1 + delta_ad)/h_d^2 (K_d x M x M) u_a
//                             + sum_{b != a} 1/(h_a h_b) (A_b x B_a x M) u_b ].
// ------------------------------------------------------------------------------------------------
template <typename T, typename R, int K>
__global__ void __launch_bounds__(128, std::is_same<R, df64>::value ? 3 : 4) box_visc_kernel(MeshView<T> m, const T *__restrict__ u, T *__restrict__ y, int cpb,
                                                       int j0, int nrows) {
  constexpr int n = K + 1, n2 = n * n, n3 = n2 * n;
  constexpr int WS = (4 * n3 > 36 * n2) ? 4 * n3 : 36 * n2;   // scratch per cell
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *U = reinterpret_cast<R *>(smem_raw);   // cpb x 3 x n3
  R *Y = U + cpb * 3 * n3;                   // cpb x 3 x n3
  R *S = Y + cpb * 3 * n3;                   // cpb x WS
  __shared__ R sc[64];                       // row scalars (one division each, done once per CTA)
  const VecConst<R> &C = vconst<R>(K);
  const int tid = threadIdx.x, nt = blockDim.x;
  const BoxBlock bk = box_block(m, cpb, j0, nrows);
  for (int t = tid; t < cpb * 3 * n3; t += nt) U[t] = r_load<R>(u[(size_t)bk.c0 * 3 * n3 + t]);
  for (int ti = tid; ti < 51; ti += nt) {
    // [5a + 0..2]: nu V (1 + delta_ad) / h_d^2; [5a + 3, 4]: nu V / (h_a h_b) for the two other
    // components b; [15 + 12 d + ...]: 1/h_d, 2/h_d, 1/h_t1, 1/h_t2, then per face s: 1/h'_d (the
    // neighbour's spacing), -nu sgn |F| / 2, nu sgn |F| / 2, tau_F nu |F|
    const double nu = (double)m.visc;
    const double hy = (double)m.hy[bk.j];
    auto hd = [&](int e) { return e == 0 ? (double)m.hx : (e == 1 ? hy : (double)m.hz); };
    const double V = (double)m.hx * hy * (double)m.hz;
    double v = 0.0;
    if (ti < 15) {
      const int a = ti / 5, k = ti % 5;
      if (k < 3) v = nu * V * (a == k ? 2.0 : 1.0) / (hd(k) * hd(k));
      else {
        const int b = k == 3 ? (a == 0 ? 1 : 0) : (a == 2 ? 1 : 2);
        v = nu * V / (hd(a) * hd(b));
      }
    } else {
      const int d = (ti - 15) / 12, k = (ti - 15) % 12;
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      const double area = V / hd(d);
      if (k == 0) v = 1.0 / hd(d);
      else if (k == 1) v = 2.0 / hd(d);
      else if (k == 2) v = 1.0 / hd(t1);
      else if (k == 3) v = 1.0 / hd(t2);
      else {
        const int s = k & 1;
        const double sgn = s ? 1.0 : -1.0;
        const int jn = bk.j + (s ? 1 : -1);
        const bool wall = d == 1 && (jn < 0 || jn >= m.ny);
        if (k < 6) v = 1.0 / ((d == 1 && !wall) ? (double)m.hy[jn] : hd(d));
        else if (k < 8) v = -0.5 * nu * sgn * area;
        else if (k < 10) v = 0.5 * nu * sgn * area;
        else {
          const double tc = (double)m.tau[bk.c0];
          const double tauF = wall ? 10.0 * tc : (d == 1 ? fmax(tc, (double)m.tau[bk.c0 + (s ? m.nx : -m.nx)]) : tc);
          v = tauF * nu * area;
        }
      }
    }
    sc[ti] = r_from_double<R>(v);
  }
  __syncthreads();
  const bool line = tid < cpb * n2;
  const int cl = line ? tid / n2 : 0, l = line ? tid - cl * n2 : 0;
  R *Uc = U + cl * 3 * n3, *Yc = Y + cl * 3 * n3, *Sc = S + cl * WS;

  // ---- volume, one output component per sweep (x-, y-, z-lines)
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int b1 = a == 0 ? 1 : 0, b2 = a == 2 ? 1 : 2;   // the other two components
    // diagonal coefficients nu V (1 + delta_ad) / h_d^2 and cross coefficients nu V / (h_a h_b)
    const R cd0 = sc[5 * a], cd1 = sc[5 * a + 1], cd2 = sc[5 * a + 2];
    const R cx1 = sc[5 * a + 3], cx2 = sc[5 * a + 4];
    // 1-D factor of cross term (a <- b) along direction e: A where e = b, B (= A^T) where e = a,
    // M otherwise
    auto xfac = [&](int b, int e, const R (&in)[n], R (&out)[n]) {
      if (e == b) mv_A<R, n>(C, in, out);
      else if (e == a) mv_AT<R, n>(C, in, out);
      else mv_M<R, n>(C, in, out);
    };
    if (line) {   // x: S0 = K_x u_a, S1 = M_x u_a, S2 = X_x u_b1, S3 = X_x u_b2
      int base, st;
      line_geom<n>(0, l, base, st);
      R v[n], o[n];
      load_line<R, n>(Uc + a * n3 + base, st, v);
      mv_K<R, n>(C, v, o);
      store_line<R, n>(Sc + base, st, o);
      mv_M<R, n>(C, v, o);
      store_line<R, n>(Sc + n3 + base, st, o);
      load_line<R, n>(Uc + b1 * n3 + base, st, v);
      xfac(b1, 0, v, o);
      store_line<R, n>(Sc + 2 * n3 + base, st, o);
      load_line<R, n>(Uc + b2 * n3 + base, st, v);
      xfac(b2, 0, v, o);
      store_line<R, n>(Sc + 3 * n3 + base, st, o);
    }
    __syncthreads();
    if (line) {   // y: W = cd0 M_y S0 + cd1 K_y S1, T = M_y S1, cross arrays
      int base, st;
      line_geom<n>(1, l, base, st);
      R s0[n], s1[n], s2[n], s3[n], w[n], t[n], x1[n], x2[n];
      load_line<R, n>(Sc + base, st, s0);
      load_line<R, n>(Sc + n3 + base, st, s1);
      load_line<R, n>(Sc + 2 * n3 + base, st, s2);
      load_line<R, n>(Sc + 3 * n3 + base, st, s3);
#pragma unroll
      for (int r = 0; r < n; ++r) w[r] = r_zero<R>();
      mva_M<R, n>(C, cd0, s0, w);
      mva_K<R, n>(C, cd1, s1, w);
      mv_M<R, n>(C, s1, t);
      xfac(b1, 1, s2, x1);
      xfac(b2, 1, s3, x2);
      // fold the cross terms whose z-factor is M into W (scaled), keep the others apart
#pragma unroll
      for (int r = 0; r < n; ++r) {
        x1[r] = cx1 * x1[r];
        x2[r] = cx2 * x2[r];
      }
      if (a == 2) {   // both cross terms take B along z
#pragma unroll
        for (int r = 0; r < n; ++r) x1[r] = x1[r] + x2[r];
      } else {        // b1 takes M along z, b2 = 2 takes A along z
#pragma unroll
        for (int r = 0; r < n; ++r) w[r] = w[r] + x1[r];
      }
      store_line<R, n>(Sc + base, st, w);
      store_line<R, n>(Sc + n3 + base, st, t);
      store_line<R, n>(Sc + 2 * n3 + base, st, a == 2 ? x1 : x2);
    }
    __syncthreads();
    if (line) {   // z: y_a = M_z W + cd2 K_z T + (B_z | A_z) X
      int base, st;
      line_geom<n>(2, l, base, st);
      R w[n], t[n], x[n], o[n], o2[n];
      load_line<R, n>(Sc + base, st, w);
      load_line<R, n>(Sc + n3 + base, st, t);
      load_line<R, n>(Sc + 2 * n3 + base, st, x);
      mv_M<R, n>(C, w, o);
      mva_K<R, n>(C, cd2, t, o);
      if (a == 2) mv_AT<R, n>(C, x, o2);
      else mv_A<R, n>(C, x, o2);
#pragma unroll
      for (int r = 0; r < n; ++r) o[r] = o[r] + o2[r];
      store_line<R, n>(Yc + a * n3 + base, st, o);
    }
    __syncthreads();
  }

  // ---- faces, one direction (both faces) at a time
  R *FU = Sc;               // [s][n2] own trace of u_d
  R *FN = FU + 2 * n2;      // [s][n2] neighbour trace of u_d
  R *FC = FN + 2 * n2;      // [s][8][n2] coefficients: C0 (3), Cn (3), Ct1, Ct2
  R *FP = FC + 16 * n2;     // [s][8][n2] after the t1-pass
  const int c = bk.c0 + cl;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int t1, t2;
    face_axes(d, t1, t2);
    const int i1 = l % n, i2 = l / n;
    int base, st;
    line_geom<n>(d, l, base, st);
    const R *scd = sc + 15 + 12 * d;
    // own and neighbour traces and physical normal derivatives at this face node (both faces)
    R Uo[2][3], Nb[2][3], G[2][3], Gn[2][3];
    int nbs[2];
    if (line) {
#pragma unroll
      for (int s = 0; s < 2; ++s) nbs[s] = neighbour(m, c, 2 * d + s);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        R v[n];
        load_line<R, n>(Uc + a * n3 + base, st, v);
        const R ih = scd[0];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          Uo[s][a] = v[s ? n - 1 : 0];
          R g = r_zero<R>();
#pragma unroll
          for (int b = 0; b < n; ++b) g = r_fma(C.de[s][b], v[b], g);
          G[s][a] = ih * g;
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          if (nbs[s] >= 0) {
            R w[n];
            neighbour_line<T, R, n>(U, u, nbs[s], bk, cpb, 3, a, base, st, w);
            Nb[s][a] = w[s ? 0 : n - 1];
            R g = r_zero<R>();
#pragma unroll
            for (int b = 0; b < n; ++b) g = r_fma(C.de[1 - s][b], w[b], g);
            Gn[s][a] = scd[4 + s] * g;
          } else {   // mirror state on a no-slip wall: u+ = -u-, grad u+ = grad u-
            Nb[s][a] = -Uo[s][a];
            Gn[s][a] = G[s][a];
          }
        }
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        FU[s * n2 + l] = Uo[s][d];
        FN[s * n2 + l] = Nb[s][d];
      }
      // an enriched neighbour across a y-face: its u~ enters the jumps (penalty and adjoint terms);
      // the flux average keeps the polynomial gradients (FN above is the polynomial trace)
      if (d == 1) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int eb = nbs[s] >= 0 ? m.enr[nbs[s]] : -1;
          if (eb >= 0) {
            R g[3];
            enr_face_nodal<T, R, n, 3>(C, m, u, eb, s, 0, i1, i2, g);
#pragma unroll
            for (int a = 0; a < 3; ++a) Nb[s][a] = Nb[s][a] + g[a];
          }
        }
      }
    }
    __syncthreads();
    if (line) {
      const R ih1 = scd[2], ih2 = scd[3];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        // tangential derivatives of the normal component's traces (wall: the neighbour's gradient
        // is the own one)
        R To1 = r_zero<R>(), To2 = r_zero<R>(), Tn1 = r_zero<R>(), Tn2 = r_zero<R>();
#pragma unroll
        for (int r = 0; r < n; ++r) {
          To1 = r_fma(C.Dg[i1 * n + r], FU[s * n2 + r + n * i2], To1);
          To2 = r_fma(C.Dg[i2 * n + r], FU[s * n2 + i1 + n * r], To2);
          Tn1 = r_fma(C.Dg[i1 * n + r], FN[s * n2 + r + n * i2], Tn1);
          Tn2 = r_fma(C.Dg[i2 * n + r], FN[s * n2 + i1 + n * r], Tn2);
        }
        To1 = ih1 * To1; To2 = ih2 * To2; Tn1 = ih1 * Tn1; Tn2 = ih2 * Tn2;
        if (nbs[s] < 0) { Tn1 = To1; Tn2 = To2; }
        const R hc = scd[6 + s];    // consistency
        const R ac = scd[8 + s];    // adjoint
        const R pc = scd[10 + s];   // penalty
        R *Fc = FC + s * 8 * n2;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const R To = a == t1 ? To1 : To2, Tn = a == t1 ? Tn1 : Tn2;
          const R So = G[s][a] + (a == d ? G[s][d] : To);
          const R Sn = Gn[s][a] + (a == d ? Gn[s][d] : Tn);
          const R J = Uo[s][a] - Nb[s][a];
          Fc[a * n2 + l] = r_fma(hc, So + Sn, pc * J);
          Fc[(3 + a) * n2 + l] = scd[a == d ? 1 : 0] * (ac * J);
        }
        Fc[6 * n2 + l] = ih1 * (ac * (Uo[s][t1] - Nb[s][t1]));
        Fc[7 * n2 + l] = ih2 * (ac * (Uo[s][t2] - Nb[s][t2]));
      }
    }
    __syncthreads();
    if (line) {   // along t1: M for C0, Cn, Ct2; A for Ct1
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const R *Fc = FC + s * 8 * n2;
        R *Fp = FP + s * 8 * n2;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const R *Mat = k == 6 ? C.A : C.M;
          R acc = r_zero<R>();
#pragma unroll
          for (int r = 0; r < n; ++r) acc = r_fma(Mat[i1 * n + r], Fc[k * n2 + r + n * i2], acc);
          Fp[k * n2 + l] = acc;
        }
      }
    }
    __syncthreads();
    if (line) {   // along t2: M (A for Ct2), then add to the own d-line
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const R *Fp = FP + s * 8 * n2;
        R z[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const R *Mat = k == 7 ? C.A : C.M;
          R acc = r_zero<R>();
#pragma unroll
          for (int r = 0; r < n; ++r) acc = r_fma(Mat[i2 * n + r], Fp[k * n2 + i1 + n * r], acc);
          z[k] = acc;
        }
        const int lay = s ? n - 1 : 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          R *ya = Yc + a * n3 + base;
#pragma unroll
          for (int mm = 0; mm < n; ++mm) ya[mm * st] = r_fma(C.de[s][mm], z[3 + a], ya[mm * st]);
          ya[lay * st] = ya[lay * st] + z[a];
        }
        Yc[d * n3 + base + lay * st] = Yc[d * n3 + base + lay * st] + (z[6] + z[7]);
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < cpb * 3 * n3; t += nt) y[(size_t)bk.c0 * 3 * n3 + t] = r_store<T>(Y[t]);
}

// ------------------------------------------------------------------------------------------------
// Volume-only operators of standard cells, exact with the k+1 Gauss points, as Kronecker products of
// 1-D node matrices (no face terms, so every row without enrichment slots qualifies):
//   OP_MASS   y_a = V (M x M x M) u_a                                        (Sec. 4.2 mass term)
//   OP_DIVDIV y_a = tau_D V sum_b 1/(h_a h_b) F_ab u_b                        (eq. div-div)
// with F_aa = K along a and M along the other two, and for b != a: A along a (the test function
// differentiated), A^T along b (the trial function differentiated), M along the third.
// ------------------------------------------------------------------------------------------------
template <typename R, int n>
__device__ __forceinline__ void divdiv_factor(const VecConst<R> &C, int a, int b, int e, const R (&in)[n], R (&out)[n]) {
  if (a == b) {
    if (e == a) mv_K<R, n>(C, in, out);
    else mv_M<R, n>(C, in, out);
  } else if (e == a) {
    mv_A<R, n>(C, in, out);
  } else if (e == b) {
    mv_AT<R, n>(C, in, out);
  } else {
    mv_M<R, n>(C, in, out);
  }
}

template <typename T, typename R, int K, int OP>
__global__ void __launch_bounds__(128) box_vol_kernel(MeshView<T> m, const T *__restrict__ u, T *__restrict__ y, int cpb,
                                                      int j0, int nrows) {
  constexpr int n = K + 1, n2 = n * n, n3 = n2 * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *U = reinterpret_cast<R *>(smem_raw);   // cpb x 3 x n3
  R *Y = U + cpb * 3 * n3;                   // cpb x 3 x n3
  R *S = Y + cpb * 3 * n3;                   // cpb x 3 x n3 scratch
  __shared__ R sc[9];                        // V (mass) or V / (h_a h_b) (div-div), [3 a + b]
  const VecConst<R> &C = vconst<R>(K);
  const int tid = threadIdx.x, nt = blockDim.x;
  const BoxBlock bk = box_block(m, cpb, j0, nrows);
  for (int t = tid; t < cpb * 3 * n3; t += nt) U[t] = r_load<R>(u[(size_t)bk.c0 * 3 * n3 + t]);
  if (tid < 9) {
    const double hd[3] = {(double)m.hx, (double)m.hy[bk.j], (double)m.hz};
    const double V = hd[0] * hd[1] * hd[2];
    sc[tid] = r_from_double<R>(OP == OP_MASS ? V : V / (hd[tid / 3] * hd[tid % 3]));
  }
  __syncthreads();
  const bool line = tid < cpb * n2;
  const int cl = line ? tid / n2 : 0, l = line ? tid - cl * n2 : 0;
  R *Uc = U + cl * 3 * n3, *Yc = Y + cl * 3 * n3, *Sc = S + cl * 3 * n3;
  if constexpr (OP == OP_MASS) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {   // x, y, z passes over the three components
      if (line) {
        int base, st;
        line_geom<n>(d, l, base, st);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          R v[n], o[n];
          load_line<R, n>((d == 0 ? Uc : Sc) + a * n3 + base, st, v);
          mv_M<R, n>(C, v, o);
          if (d == 2) {
#pragma unroll
            for (int r = 0; r < n; ++r) o[r] = sc[0] * o[r];
          }
          store_line<R, n>((d == 2 ? Yc : Sc) + a * n3 + base, st, o);
        }
      }
      __syncthreads();
    }
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) {   // one output component per sweep; S[b] holds F_ab u_b pass by pass
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (line) {
          int base, st;
          line_geom<n>(d, l, base, st);
          R acc[n];
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            R v[n], o[n];
            load_line<R, n>((d == 0 ? Uc : Sc) + b * n3 + base, st, v);
            divdiv_factor<R, n>(C, a, b, d, v, o);
            if (d < 2) {
              store_line<R, n>(Sc + b * n3 + base, st, o);
            } else {
#pragma unroll
              for (int r = 0; r < n; ++r) acc[r] = b == 0 ? sc[3 * a] * o[r] : r_fma(sc[3 * a + b], o[r], acc[r]);
            }
          }
          if (d == 2) store_line<R, n>(Yc + a * n3 + base, st, acc);
        }
        __syncthreads();
      }
    }
  }
  if constexpr (OP == OP_MASS) {
    for (int t = tid; t < cpb * 3 * n3; t += nt) y[(size_t)bk.c0 * 3 * n3 + t] = r_store<T>(Y[t]);
  } else {
    for (int t = tid; t < cpb * 3 * n3; t += nt) {
      const int c = bk.c0 + t / (3 * n3);
      y[(size_t)bk.c0 * 3 * n3 + t] = r_store<T>(r_load<R>(m.tau_d[c]) * Y[t]);
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Convective term F^c(v, u) of standard cells (Sec. 4.2): -(grad v, u x u)_K + (v, F*.n)_dK with the
// local Lax-Friedrichs flux F* = 1/2 (u^- (u^-.n) + u^+ (u^+.n)) + Lambda/2 (u^- - u^+),
// Lambda = max(2|u^-.n|, 2|u^+.n|), u^+ = -u^- on walls. The integrand is not a polynomial of the
// nodal degree (the flux has |.| and max), so it is evaluated at the operator's own
// q = floor(3k/2) + 1 Gauss points per direction (Sec. 4.4), by sum factorisation in point space:
// values of the three components at the q^3 points, the nine products u_a u_d, integration against
// d phi / d x_d; on each face the traces of both sides at q x q points, the flux, integration back
// to the face layer. Passes assign whole lines to threads (a thread may take several lines).
// ------------------------------------------------------------------------------------------------
template <int n, int q>
struct ConvPlan {
  static constexpr int n2 = n * n, n3 = n2 * n, q2 = q * q, q3 = q2 * q;
  static constexpr int A1 = (3 * q * n2 > 3 * q2 * n) ? 3 * q * n2 : 3 * q2 * n;   // fwd x / bwd z (one output)
  static constexpr int A2 = (3 * q2 * n > 2 * q * n2) ? 3 * q2 * n : 2 * q * n2;   // fwd y / bwd y (one output)
  static constexpr int FACE = 12 * n2 + 12 * q * n + 12 * q2 + 6 * q2 + 6 * q * n;
  static constexpr int WORK = (3 * q3 + A1 + A2 > FACE) ? 3 * q3 + A1 + A2 : FACE;
  static constexpr int PER_CELL = 3 * n3 + 3 * n3 + WORK;   // U, Y, work
};

template <typename T, typename R, int K>
__global__ void __launch_bounds__(128) box_conv_kernel(MeshView<T> m, const T *__restrict__ u, T *__restrict__ y, int cpb,
                                                       int j0, int nrows) {
  constexpr int n = K + 1, n2 = n * n, n3 = n2 * n;
  constexpr int q = (3 * K) / 2 + 1, q2 = q * q, q3 = q2 * q;
  using P = ConvPlan<n, q>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *U = reinterpret_cast<R *>(smem_raw);   // cpb x 3 x n3
  R *Y = U + cpb * 3 * n3;                   // cpb x 3 x n3
  R *W = Y + cpb * 3 * n3;                   // cpb x WORK
  __shared__ R sc[6];                        // -V/h_d (volume), V/h_d (face area)
  const VecConst<R> &C = vconst<R>(K);
  const int tid = threadIdx.x, nt = blockDim.x;
  const BoxBlock bk = box_block(m, cpb, j0, nrows);
  for (int t = tid; t < cpb * 3 * n3; t += nt) {
    U[t] = r_load<R>(u[(size_t)bk.c0 * 3 * n3 + t]);
    Y[t] = r_zero<R>();
  }
  if (tid < 6) {
    const double hy = (double)m.hy[bk.j];
    const double V = (double)m.hx * hy * (double)m.hz;
    const int d = tid % 3;
    const double h = d == 0 ? (double)m.hx : (d == 1 ? hy : (double)m.hz);
    sc[tid] = r_from_double<R>((tid < 3 ? -1.0 : 1.0) * V / h);
  }
  __syncthreads();
  auto Wc = [&](int cl) { return W + cl * P::WORK; };
  // ---- volume: values at the points (x: n -> q, then y, then z)
  for (int t = tid; t < cpb * 3 * n2; t += nt) {
    const int cl = t / (3 * n2), r = t - cl * 3 * n2, a = r / n2, l = r - a * n2;
    R v[n];
    load_line<R, n>(U + (cl * 3 + a) * n3 + n * l, 1, v);
    R *out = Wc(cl) + 3 * q3 + a * q * n2 + q * l;
    R o[q];
    interp_eo<R, n, q>(C, v, o);
#pragma unroll
    for (int i = 0; i < q; ++i) out[i] = o[i];
  }
  __syncthreads();
  for (int t = tid; t < cpb * 3 * q * n; t += nt) {   // lines (i0, i2), i0 < q, i2 < n
    const int cl = t / (3 * q * n), r = t - cl * 3 * q * n, a = r / (q * n), l = r - a * q * n;
    const int i0 = l % q, i2 = l / q;
    R v[n];
    load_line<R, n>(Wc(cl) + 3 * q3 + a * q * n2 + i0 + q * n * i2, q, v);
    R *out = Wc(cl) + 3 * q3 + P::A1 + a * q2 * n + i0 + q2 * i2;
    R o[q];
    interp_eo<R, n, q>(C, v, o);
#pragma unroll
    for (int i = 0; i < q; ++i) out[q * i] = o[i];
  }
  __syncthreads();
  for (int t = tid; t < cpb * 3 * q2; t += nt) {   // lines (i0, i1)
    const int cl = t / (3 * q2), r = t - cl * 3 * q2, a = r / q2, l = r - a * q2;
    R v[n];
    load_line<R, n>(Wc(cl) + 3 * q3 + P::A1 + a * q2 * n + l, q2, v);
    R *out = Wc(cl) + a * q3 + l;
    R o[q];
    interp_eo<R, n, q>(C, v, o);
#pragma unroll
    for (int i = 0; i < q; ++i) out[q2 * i] = o[i];
  }
  __syncthreads();
  // ---- volume: -sum_d (V/h_d) sum_points w (d phi / d xi_d) u_a u_d, one output component at a time
  for (int a = 0; a < 3; ++a) {
    for (int t = tid; t < cpb * q2; t += nt) {   // z-lines (i0, i1): F_ad along z, integrate along z
      const int cl = t / q2, l = t - cl * q2, i0 = l % q, i1 = l / q;
      const R *V = Wc(cl);
      R z0[n], z1[n], z2[n];
      R F0[q], F1[q], F2[q];
      const R w01 = C.wc[i0] * C.wc[i1];
#pragma unroll
      for (int j = 0; j < q; ++j) {
        const int pt = l + q2 * j;
        const R ua = V[a * q3 + pt];
        const R wa = (w01 * C.wc[j]) * ua;
        F0[j] = sc[0] * (wa * V[pt]);            // F_a0 = -(V/h_x) w u_a u_x
        F1[j] = sc[1] * (wa * V[q3 + pt]);
        F2[j] = sc[2] * (wa * V[2 * q3 + pt]);
      }
      {
        constexpr int qh = q / 2 > 0 ? q / 2 : 1;
        R fe[qh], fo[qh];
        point_eo<R, q>(F2, fe, fo);
        tinterp_d_eo<R, n, q, false>(C, fe, fo, F2[q / 2], z0);   // D_z^T F_a2
        point_eo<R, q>(F1, fe, fo);
        tinterp_s_eo<R, n, q, false>(C, fe, fo, F1[q / 2], z1);   // S_z^T F_a1
        point_eo<R, q>(F0, fe, fo);
        tinterp_s_eo<R, n, q, false>(C, fe, fo, F0[q / 2], z2);   // S_z^T F_a0
      }
      R *Z = Wc(cl) + 3 * q3;
      store_line<R, n>(Z + l, q2, z0);
      store_line<R, n>(Z + q2 * n + l, q2, z1);
      store_line<R, n>(Z + 2 * q2 * n + l, q2, z2);
    }
    __syncthreads();
    for (int t = tid; t < cpb * q * n; t += nt) {   // y-lines (i0, m): Y0 = S_y^T Z0 + D_y^T Z1, Y1 = S_y^T Z2
      const int cl = t / (q * n), l = t - cl * q * n, i0 = l % q, mz = l / q;
      const R *Z = Wc(cl) + 3 * q3;
      R y0[n], y1[n];
      R za[q], zb[q], zc[q];
#pragma unroll
      for (int j = 0; j < q; ++j) {
        const int pt = i0 + q * j + q2 * mz;
        za[j] = Z[pt];
        zb[j] = Z[q2 * n + pt];
        zc[j] = Z[2 * q2 * n + pt];
      }
      {
        constexpr int qh = q / 2 > 0 ? q / 2 : 1;
        R fe[qh], fo[qh];
        point_eo<R, q>(za, fe, fo);
        tinterp_s_eo<R, n, q, false>(C, fe, fo, za[q / 2], y0);
        point_eo<R, q>(zb, fe, fo);
        tinterp_d_eo<R, n, q, true>(C, fe, fo, zb[q / 2], y0);
        point_eo<R, q>(zc, fe, fo);
        tinterp_s_eo<R, n, q, false>(C, fe, fo, zc[q / 2], y1);
      }
      R *Yb = Wc(cl) + 3 * q3 + P::A1;
      store_line<R, n>(Yb + i0 + q * n * mz, q, y0);
      store_line<R, n>(Yb + q * n2 + i0 + q * n * mz, q, y1);
    }
    __syncthreads();
    for (int t = tid; t < cpb * n2; t += nt) {   // x-lines (b, m): y_a = S_x^T Y0 + D_x^T Y1
      const int cl = t / n2, l = t - cl * n2;
      const R *Yb = Wc(cl) + 3 * q3 + P::A1 + q * l;
      R o[n];
      R ya[q], yb[q];
#pragma unroll
      for (int j = 0; j < q; ++j) { ya[j] = Yb[j]; yb[j] = Yb[q * n2 + j]; }
      {
        constexpr int qh = q / 2 > 0 ? q / 2 : 1;
        R fe[qh], fo[qh];
        point_eo<R, q>(ya, fe, fo);
        tinterp_s_eo<R, n, q, false>(C, fe, fo, ya[q / 2], o);
        point_eo<R, q>(yb, fe, fo);
        tinterp_d_eo<R, n, q, true>(C, fe, fo, yb[q / 2], o);
      }
      R *yo = Y + (cl * 3 + a) * n3 + n * l;
#pragma unroll
      for (int b = 0; b < n; ++b) yo[b] = o[b];
    }
    __syncthreads();
  }
  // ---- faces, one direction (both faces) at a time: slots k = (s * 2 + side) * 3 + a
  for (int d = 0; d < 3; ++d) {
    int t1, t2;
    face_axes(d, t1, t2);
    // layer values of both sides (side 0: own layer at xi_d = s; side 1: the neighbour's opposite
    // layer; walls leave side 1 unused, the mirror state is taken at the flux)
    for (int t = tid; t < cpb * 12 * n2; t += nt) {
      const int cl = t / (12 * n2), r = t - cl * 12 * n2, k = r / n2, l = r - k * n2;
      const int a = k % 3, side = (k / 3) & 1, s = k / 6;
      const int i1 = l % n, i2 = l / n;
      R val = r_zero<R>();
      if (side == 0) {
        val = U[(cl * 3 + a) * n3 + node_index(d, t1, t2, s ? n - 1 : 0, i1, i2, n)];
      } else {
        const int nb = neighbour(m, bk.c0 + cl, 2 * d + s);
        if (nb >= 0) {
          const int idx = node_index(d, t1, t2, s ? 0 : n - 1, i1, i2, n);
          const int rel = nb - bk.c0;
          val = (rel >= 0 && rel < cpb) ? U[(rel * 3 + a) * n3 + idx] : r_load<R>(u[((size_t)nb * 3 + a) * n3 + idx]);
        }
      }
      Wc(cl)[k * n2 + l] = val;
    }
    __syncthreads();
    for (int t = tid; t < cpb * 12 * n; t += nt) {   // along t1: n -> q
      const int cl = t / (12 * n), r = t - cl * 12 * n, k = r / n, i2 = r - k * n;
      R v[n];
      load_line<R, n>(Wc(cl) + k * n2 + n * i2, 1, v);
      R *out = Wc(cl) + 12 * n2 + k * q * n + q * i2;
      R o[q];
      interp_eo<R, n, q>(C, v, o);
#pragma unroll
      for (int i = 0; i < q; ++i) out[i] = o[i];
    }
    __syncthreads();
    for (int t = tid; t < cpb * 12 * q; t += nt) {   // along t2: n -> q
      const int cl = t / (12 * q), r = t - cl * 12 * q, k = r / q, j1 = r - k * q;
      R v[n];
      load_line<R, n>(Wc(cl) + 12 * n2 + k * q * n + j1, q, v);
      R *out = Wc(cl) + 12 * n2 + 12 * q * n + k * q2 + j1;
      R o[q];
      interp_eo<R, n, q>(C, v, o);
#pragma unroll
      for (int i = 0; i < q; ++i) out[q * i] = o[i];
    }
    __syncthreads();
    for (int t = tid; t < cpb * 2 * q2; t += nt) {   // local Lax-Friedrichs flux at the face points
      const int cl = t / (2 * q2), r = t - cl * 2 * q2, s = r / q2, pt = r - s * q2;
      const R *Tr = Wc(cl) + 12 * n2 + 12 * q * n;
      const bool wall = neighbour(m, bk.c0 + cl, 2 * d + s) < 0;
      R um[3], up[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        um[a] = Tr[((s * 2 + 0) * 3 + a) * q2 + pt];
        up[a] = wall ? -um[a] : Tr[((s * 2 + 1) * 3 + a) * q2 + pt];
      }
      const int eb = (d == 1 && !wall) ? m.enr[neighbour(m, bk.c0 + cl, 2 + s)] : -1;
      if (eb >= 0) {   // the enriched neighbour's u~ at the point (psi from its convective wall table)
        const R psi = r_load<R>(m.wt_face[1][(((size_t)eb * 6 + 2 + (1 - s)) * m.fpmax[1] + pt) * WT]);
        const R x = C.xc[pt % q], z = C.xc[pt / q];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          R e4[4];
          enr_face_coeffs<T, R>(m, u, eb, s, a, e4);
          up[a] = r_fma(psi, enr_face_sum<R>(e4, m.nef == 1, x, z), up[a]);
        }
      }
      const R umd = d == 0 ? um[0] : (d == 1 ? um[1] : um[2]);
      const R upd = d == 0 ? up[0] : (d == 1 ? up[1] : up[2]);
      const R unm = s ? umd : -umd, unp = s ? upd : -upd;
      // Lambda / 2 = max(|u^-.n|, |u^+.n|)
      const R lam = r_abs_ge(unm, unp) ? r_abs(unm) : r_abs(unp);
      const R wq = sc[3 + d] * (C.wc[pt % q] * C.wc[pt / q]);
      R *Fl = Wc(cl) + 12 * n2 + 12 * q * n + 12 * q2;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        // 1/2 (u^-_a (u^-.n) + u^+_a (u^+.n)) + (Lambda/2)(u^-_a - u^+_a), Lambda/2 = max(|u^-.n|, |u^+.n|)
        const R F = r_fma(lam, um[a] - up[a], r_half<R>() * r_fma(um[a], unm, up[a] * unp));
        Fl[(s * 3 + a) * q2 + pt] = wq * F;
      }
    }
    __syncthreads();
    for (int t = tid; t < cpb * 6 * q; t += nt) {   // back along t2: q -> n
      const int cl = t / (6 * q), r = t - cl * 6 * q, k = r / q, j1 = r - k * q;
      const R *Fl = Wc(cl) + 12 * n2 + 12 * q * n + 12 * q2 + k * q2;
      R o[n], f[q];
#pragma unroll
      for (int j = 0; j < q; ++j) f[j] = Fl[j1 + q * j];
      {
        constexpr int qh = q / 2 > 0 ? q / 2 : 1;
        R fe[qh], fo[qh];
        point_eo<R, q>(f, fe, fo);
        tinterp_s_eo<R, n, q, false>(C, fe, fo, f[q / 2], o);
      }
      R *Bt = Wc(cl) + 12 * n2 + 12 * q * n + 18 * q2 + k * q * n;
      store_line<R, n>(Bt + j1, q, o);
    }
    __syncthreads();
    for (int t = tid; t < cpb * 6 * n; t += nt) {   // back along t1: q -> n, add to the face layer
      const int cl = t / (6 * n), r = t - cl * 6 * n, k = r / n, i2 = r - k * n;
      const int s = k / 3, a = k % 3;
      const R *Bt = Wc(cl) + 12 * n2 + 12 * q * n + 18 * q2 + k * q * n + q * i2;
      R o[n], f[q];
#pragma unroll
      for (int j = 0; j < q; ++j) f[j] = Bt[j];
      {
        constexpr int qh = q / 2 > 0 ? q / 2 : 1;
        R fe[qh], fo[qh];
        point_eo<R, q>(f, fe, fo);
        tinterp_s_eo<R, n, q, false>(C, fe, fo, f[q / 2], o);
      }
      R *ya = Y + (cl * 3 + a) * n3;
#pragma unroll
      for (int b = 0; b < n; ++b) {
        const int idx = node_index(d, t1, t2, s ? n - 1 : 0, b, i2, n);
        ya[idx] = ya[idx] + o[b];
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < cpb * 3 * n3; t += nt) y[(size_t)bk.c0 * 3 * n3 + t] = r_store<T>(Y[t]);
}

// ------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------

cudaError_t box_vec_constants_init() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
  static VecConst<double> h64[5];
  static VecConst<float> h32[5];
  static VecConst<df64> hdf[5];
  std::memset(h64, 0, sizeof(h64));
  for (int k = 1; k <= 5; ++k) {
    VecConst<double> &V = h64[k - 1];
    Basis<double> B;
    fill_basis<double>(k, (3 * k) / 2 + 1, k + 1, &B);
    const int n = k + 1, q = B.q[QSET_LIN];
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        double mv = 0.0, kv = 0.0, av = 0.0;
        for (int t = 0; t < q; ++t) {
          const double w = B.w[QSET_LIN][t];
          mv += w * B.S[QSET_LIN][t * n + a] * B.S[QSET_LIN][t * n + b];
          kv += w * B.D[QSET_LIN][t * n + a] * B.D[QSET_LIN][t * n + b];
          av += w * B.D[QSET_LIN][t * n + a] * B.S[QSET_LIN][t * n + b];
        }
        V.M[a * n + b] = mv;
        V.K[a * n + b] = kv;
        V.A[a * n + b] = av;
      }
    double z[NMAX];
    lobatto_nodes(n, z);
    for (int i = 0; i < n; ++i) {
      double val[NMAX], der[NMAX];
      lagrange_row(n, z, z[i], val, der);
      for (int j = 0; j < n; ++j) V.Dg[i * n + j] = der[j];
    }
    for (int s = 0; s < 2; ++s)
      for (int j = 0; j < n; ++j) V.de[s][j] = B.dend[s][j];
    const int qc = B.q[QSET_CONV];
    for (int t = 0; t < qc; ++t) {
      for (int j = 0; j < n; ++j) {
        V.Sc[t * n + j] = B.S[QSET_CONV][t * n + j];
        V.Dc[t * n + j] = B.D[QSET_CONV][t * n + j];
      }
      V.wc[t] = B.w[QSET_CONV][t];
    }
    for (int t = 0; t < qc; ++t) V.xc[t] = B.x[QSET_CONV][t];
    if (q != n) return cudaErrorInvalidValue;   // the node-space face integrals assume k+1 points
    for (int t = 0; t < n; ++t) V.xg[t] = B.x[QSET_LIN][t];
    {
      // Gauss-Jordan inverse of the n x n table S[t][b] = l_b(x_t), partial pivoting
      double a[NMAX][2 * NMAX];
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c) a[r][c] = c < n ? B.S[QSET_LIN][r * n + c] : (c - n == r ? 1.0 : 0.0);
      for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
          if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
        for (int x = 0; x < 2 * n; ++x) std::swap(a[c][x], a[piv][x]);
        const double inv = 1.0 / a[c][c];
        for (int x = 0; x < 2 * n; ++x) a[c][x] *= inv;
        for (int r = 0; r < n; ++r)
          if (r != c) {
            const double f = a[r][c];
            for (int x = 0; x < 2 * n; ++x) a[r][x] -= f * a[c][x];
          }
      }
      for (int b = 0; b < n; ++b)
        for (int t = 0; t < n; ++t) V.Sinv[b * n + t] = a[b][n + t];
    }
    for (int r = 0; r < n / 2; ++r)
      for (int b = 0; b < n / 2; ++b) {
        const int i = r * n + b, j = r * n + n - 1 - b;
        V.ME[i] = 0.5 * (V.M[i] + V.M[j]);
        V.MO[i] = 0.5 * (V.M[i] - V.M[j]);
        V.KE[i] = 0.5 * (V.K[i] + V.K[j]);
        V.KO[i] = 0.5 * (V.K[i] - V.K[j]);
        V.AE[i] = 0.5 * (V.A[i] + V.A[j]);
        V.AO[i] = 0.5 * (V.A[i] - V.A[j]);
        const double t0 = V.A[b * n + r], t1 = V.A[(n - 1 - b) * n + r];   // A^T[r][b], A^T[r][n-1-b]
        V.TE[i] = 0.5 * (t0 + t1);
        V.TO[i] = 0.5 * (t0 - t1);
      }
    for (int t = 0; t < qc / 2; ++t)
      for (int j = 0; j < n / 2; ++j) {
        const double s0 = B.S[QSET_CONV][t * n + j], s1 = B.S[QSET_CONV][t * n + n - 1 - j];
        const double d0 = B.D[QSET_CONV][t * n + j], d1 = B.D[QSET_CONV][t * n + n - 1 - j];
        V.SE[t * n + j] = 0.5 * (s0 + s1);
        V.SO[t * n + j] = 0.5 * (s0 - s1);
        V.DA[t * n + j] = 0.5 * (d0 - d1);
        V.DB[t * n + j] = 0.5 * (d0 + d1);
      }
  }
  auto split = [](double v) { const float h = (float)v; return df64{h, (float)(v - (double)h)}; };
  const double *src = reinterpret_cast<const double *>(h64);
  float *d32 = reinterpret_cast<float *>(h32);
  df64 *ddf = reinterpret_cast<df64 *>(hdf);
  static_assert(sizeof(VecConst<double>) == 2 * sizeof(VecConst<float>), "layout");
  static_assert(sizeof(VecConst<double>) == sizeof(VecConst<df64>), "layout");
  for (size_t i = 0; i < sizeof(h64) / sizeof(double); ++i) {
    d32[i] = (float)src[i];
    ddf[i] = split(src[i]);
  }
  e = cudaMemcpyToSymbol(c_vec64, h64, sizeof(h64));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_vec32, h32, sizeof(h32));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_vecdf, hdf, sizeof(hdf));
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

// cells per CTA: the largest power of two dividing nx with cpb * lines <= 128 and cpb <= 8
static int vec_cpb(int nx, int lines) {
  int c = 1;
  while (c * 2 <= 8 && (c * 2) * lines <= 128 && nx % (c * 2) == 0) c *= 2;
  return c;
}

template <typename T, typename R, int K, int OP>
static cudaError_t launch_box_op_k(const MeshView<T> &m, const T *u, T *y, int j0, int nrows, cudaStream_t s) {
  constexpr int n = K + 1, n2 = n * n, n3 = n2 * n, q = (3 * K) / 2 + 1;
  int cpb, threads;
  size_t per_cell;
  if (OP == OP_CONV) {
    cpb = vec_cpb(m.nx, q * q);
    threads = 128;
    per_cell = ConvPlan<n, q>::PER_CELL;
  } else {
    cpb = vec_cpb(m.nx, n2);
    threads = ((cpb * n2 + 31) / 32) * 32;
    per_cell = OP == OP_DIV ? 7 * n3
                            : (OP == OP_VISC ? 6 * n3 + ((4 * n3 > 36 * n2) ? 4 * n3 : 36 * n2) : 9 * n3);
  }
  const size_t sm = sizeof(R) * per_cell * cpb;
  auto kern = [] {
    if constexpr (OP == OP_DIV) return box_div_kernel<T, R, K>;
    else if constexpr (OP == OP_VISC) return box_visc_kernel<T, R, K>;
    else if constexpr (OP == OP_CONV) return box_conv_kernel<T, R, K>;
    else return box_vol_kernel<T, R, K, OP>;
  }();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (sm > 200 * 1024) return cudaErrorInvalidConfiguration;
  const int blocks = (m.nx / cpb) * nrows * m.nz;
  note_launch();
  kern<<<blocks, threads, sm, s>>>(m, u, y, cpb, j0, nrows);
  return cudaGetLastError();
}

template <typename T, typename R>
cudaError_t launch_box_vec_rows(int op, const MeshView<T> &m, const T *u, T *y, int j0, int nrows, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  cudaError_t e = box_vec_constants_init();
  if (e != cudaSuccess) return e;
  if (op == OP_DIV) {
    switch (m.n1) {
      case 2: return launch_box_op_k<T, R, 1, OP_DIV>(m, u, y, j0, nrows, s);
      case 3: return launch_box_op_k<T, R, 2, OP_DIV>(m, u, y, j0, nrows, s);
      case 4: return launch_box_op_k<T, R, 3, OP_DIV>(m, u, y, j0, nrows, s);
      case 5: return launch_box_op_k<T, R, 4, OP_DIV>(m, u, y, j0, nrows, s);
      case 6: return launch_box_op_k<T, R, 5, OP_DIV>(m, u, y, j0, nrows, s);
    }
  } else if (op == OP_VISC) {
    switch (m.n1) {
      case 2: return launch_box_op_k<T, R, 1, OP_VISC>(m, u, y, j0, nrows, s);
      case 3: return launch_box_op_k<T, R, 2, OP_VISC>(m, u, y, j0, nrows, s);
      case 4: return launch_box_op_k<T, R, 3, OP_VISC>(m, u, y, j0, nrows, s);
      case 5: return launch_box_op_k<T, R, 4, OP_VISC>(m, u, y, j0, nrows, s);
      case 6: return launch_box_op_k<T, R, 5, OP_VISC>(m, u, y, j0, nrows, s);
    }
  } else if (op == OP_CONV) {
    switch (m.n1) {
      case 2: return launch_box_op_k<T, R, 1, OP_CONV>(m, u, y, j0, nrows, s);
      case 3: return launch_box_op_k<T, R, 2, OP_CONV>(m, u, y, j0, nrows, s);
      case 4: return launch_box_op_k<T, R, 3, OP_CONV>(m, u, y, j0, nrows, s);
      case 5: return launch_box_op_k<T, R, 4, OP_CONV>(m, u, y, j0, nrows, s);
      case 6: return launch_box_op_k<T, R, 5, OP_CONV>(m, u, y, j0, nrows, s);
    }
  } else if (op == OP_MASS || op == OP_DIVDIV) {
    if constexpr (!std::is_same<R, df64>::value) {   // native precisions only
      if (op == OP_MASS) {
        switch (m.n1) {
          case 2: return launch_box_op_k<T, R, 1, OP_MASS>(m, u, y, j0, nrows, s);
          case 3: return launch_box_op_k<T, R, 2, OP_MASS>(m, u, y, j0, nrows, s);
          case 4: return launch_box_op_k<T, R, 3, OP_MASS>(m, u, y, j0, nrows, s);
          case 5: return launch_box_op_k<T, R, 4, OP_MASS>(m, u, y, j0, nrows, s);
          case 6: return launch_box_op_k<T, R, 5, OP_MASS>(m, u, y, j0, nrows, s);
        }
      } else {
        switch (m.n1) {
          case 2: return launch_box_op_k<T, R, 1, OP_DIVDIV>(m, u, y, j0, nrows, s);
          case 3: return launch_box_op_k<T, R, 2, OP_DIVDIV>(m, u, y, j0, nrows, s);
          case 4: return launch_box_op_k<T, R, 3, OP_DIVDIV>(m, u, y, j0, nrows, s);
          case 5: return launch_box_op_k<T, R, 4, OP_DIVDIV>(m, u, y, j0, nrows, s);
          case 6: return launch_box_op_k<T, R, 5, OP_DIVDIV>(m, u, y, j0, nrows, s);
        }
      }
    }
  }
  return cudaErrorInvalidValue;
}

template cudaError_t launch_box_vec_rows<double, double>(int, const MeshView<double> &, const double *, double *, int,
                                                         int, cudaStream_t);
template cudaError_t launch_box_vec_rows<float, float>(int, const MeshView<float> &, const float *, float *, int, int,
                                                       cudaStream_t);
template cudaError_t launch_box_vec_rows<double, df64>(int, const MeshView<double> &, const double *, double *, int,
                                                       int, cudaStream_t);

}  // namespace dgw
