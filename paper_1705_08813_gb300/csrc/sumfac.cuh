// CTA-cooperative sum-factorisation building blocks (Sec. 4.4: tensor-product evaluation of the
// Q_k basis at Gauss points, done here by 1-D passes in shared memory).
//
// 3-D arrays are x-fastest: index i0 + s0*(i1 + s1*i2). A 1-D matrix M is stored q x n
// (rows = points, cols = nodes). Forward passes map nodes -> points along one axis, transposed
// passes map points -> nodes (integration). Every thread walks the output with the same
// stride, so an accumulating pass issued right after a pass over the same output needs no
// barrier in between.
#pragma once

#include "dgw_internal.h"

namespace dgw {

template <typename T>
__device__ __forceinline__ void axis_pass(const T *__restrict__ in, T *__restrict__ out, int s0, int s1,
                                          int s2, int ax, const T *__restrict__ M, int n, int q,
                                          bool trans, bool acc) {
  const int mi = trans ? q : n;   // length summed over
  const int mo = trans ? n : q;   // output length along ax
  const int o0 = ax == 0 ? mo : s0, o1 = ax == 1 ? mo : s1, o2 = ax == 2 ? mo : s2;
  const int total = o0 * o1 * o2;
  const int stride = ax == 0 ? 1 : (ax == 1 ? s0 : s0 * s1);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int i0 = t % o0, i1 = (t / o0) % o1, i2 = t / (o0 * o1);
    const int r = ax == 0 ? i0 : (ax == 1 ? i1 : i2);
    const int base = (ax == 0 ? 0 : i0) + s0 * ((ax == 1 ? 0 : i1) + s1 * (ax == 2 ? 0 : i2));
    T sum = T(0);
    if (!trans) {
      const T *row = M + r * n;
      for (int c = 0; c < mi; ++c) sum += row[c] * in[base + c * stride];
    } else {
      for (int c = 0; c < mi; ++c) sum += M[c * n + r] * in[base + c * stride];
    }
    out[t] = acc ? out[t] + sum : sum;
  }
}

// Tables of one cell evaluation: per axis the value and derivative matrices and point counts.
template <typename T>
struct AxisTabs {
  const T *S[3];
  const T *D[3];
  int q[3];
};

// u (n^3 nodes) -> val, g0, g1, g2 at q0 x q1 x q2 points (reference derivatives d/dxi_d).
// Any output may be null. tmp must hold 5 * max(q0*n*n, q0*q1*n) entries.
template <typename T>
__device__ void eval_cell(const T *u, int n, const AxisTabs<T> &t, T *val, T *g0, T *g1, T *g2, T *tmp) {
  const int q0 = t.q[0], q1 = t.q[1], q2 = t.q[2];
  const int sz = max(q0 * n * n, q0 * q1 * n);
  T *X0 = tmp, *X1 = tmp + sz, *Y00 = tmp + 2 * sz, *Y01 = tmp + 3 * sz, *Y10 = tmp + 4 * sz;
  const bool need_x1 = g0 != nullptr;
  axis_pass(u, X0, n, n, n, 0, t.S[0], n, q0, false, false);
  if (need_x1) axis_pass(u, X1, n, n, n, 0, t.D[0], n, q0, false, false);
  __syncthreads();
  axis_pass(X0, Y00, q0, n, n, 1, t.S[1], n, q1, false, false);
  if (g1) axis_pass(X0, Y01, q0, n, n, 1, t.D[1], n, q1, false, false);
  if (need_x1) axis_pass(X1, Y10, q0, n, n, 1, t.S[1], n, q1, false, false);
  __syncthreads();
  if (val) axis_pass(Y00, val, q0, q1, n, 2, t.S[2], n, q2, false, false);
  if (g2) axis_pass(Y00, g2, q0, q1, n, 2, t.D[2], n, q2, false, false);
  if (g1) axis_pass(Y01, g1, q0, q1, n, 2, t.S[2], n, q2, false, false);
  if (g0) axis_pass(Y10, g0, q0, q1, n, 2, t.S[2], n, q2, false, false);
  __syncthreads();
}

// r (n^3) += sum_points [ f phi + h0 dphi/dxi0 + h1 dphi/dxi1 + h2 dphi/dxi2 ]. Inputs may be null
// (treated as zero). tmp as for eval_cell.
template <typename T>
__device__ void integrate_cell(const T *f, const T *h0, const T *h1, const T *h2, int n, const AxisTabs<T> &t,
                               T *r, T *tmp) {
  const int q0 = t.q[0], q1 = t.q[1], q2 = t.q[2];
  const int sz = max(q0 * n * n, q0 * q1 * n);
  T *Z0 = tmp, *Z1 = tmp + sz, *Z2 = tmp + 2 * sz, *Y0 = tmp + 3 * sz, *Y1 = tmp + 4 * sz;
  // z: points -> nodes
  bool z0 = false;
  if (f) { axis_pass(f, Z0, q0, q1, q2, 2, t.S[2], n, q2, true, false); z0 = true; }
  if (h2) { axis_pass(h2, Z0, q0, q1, q2, 2, t.D[2], n, q2, true, z0); z0 = true; }
  if (h1) axis_pass(h1, Z1, q0, q1, q2, 2, t.S[2], n, q2, true, false);
  if (h0) axis_pass(h0, Z2, q0, q1, q2, 2, t.S[2], n, q2, true, false);
  __syncthreads();
  bool y0 = false;
  if (z0) { axis_pass(Z0, Y0, q0, q1, n, 1, t.S[1], n, q1, true, false); y0 = true; }
  if (h1) { axis_pass(Z1, Y0, q0, q1, n, 1, t.D[1], n, q1, true, y0); y0 = true; }
  if (h0) axis_pass(Z2, Y1, q0, q1, n, 1, t.S[1], n, q1, true, false);
  __syncthreads();
  if (y0) axis_pass(Y0, r, q0, n, n, 0, t.S[0], n, q0, true, true);
  if (h0) axis_pass(Y1, r, q0, n, n, 0, t.D[0], n, q0, true, true);
  __syncthreads();
}

// Face (axis d, side s) geometry of the tensor-product cell: tangential axes t1 < t2.
__device__ __forceinline__ void face_axes(int d, int &t1, int &t2) {
  t1 = d == 0 ? 1 : 0;
  t2 = d == 2 ? 1 : 2;
}

__device__ __forceinline__ int node_index(int d, int t1, int t2, int id, int i1, int i2, int n) {
  int idx[3];
  idx[d] = id; idx[t1] = i1; idx[t2] = i2;
  return idx[0] + n * (idx[1] + n * idx[2]);
}

// Trace of u on face (d, side): at p1 x p2 face points (t1 fastest) the value, the reference
// normal derivative d/dxi_d and the tangential derivatives d/dxi_t1, d/dxi_t2 (outputs may be
// null). S1/D1 tabulate axis t1 at p1 points, S2/D2 axis t2 at p2 points. tmp: 5*n*max(n,p1).
template <typename T>
__device__ void eval_face(const T *u, int n, int d, int side, const T *dend, const T *S1, const T *D1, int p1,
                          const T *S2, const T *D2, int p2, T *val, T *gd, T *gt1, T *gt2, T *tmp) {
  int t1, t2;
  face_axes(d, t1, t2);
  const int nn = n * n;
  const int sz = n * max(n, p1);
  T *V2 = tmp, *N2 = tmp + nn, *A0 = tmp + 2 * sz, *A1 = tmp + 3 * sz, *B0 = tmp + 4 * sz;
  const int layer = side ? n - 1 : 0;
  for (int t = threadIdx.x; t < nn; t += blockDim.x) {
    const int i1 = t % n, i2 = t / n;
    V2[t] = u[node_index(d, t1, t2, layer, i1, i2, n)];
    if (gd) {
      T s = T(0);
      for (int j = 0; j < n; ++j) s += dend[j] * u[node_index(d, t1, t2, j, i1, i2, n)];
      N2[t] = s;
    }
  }
  __syncthreads();
  axis_pass(V2, A0, n, n, 1, 0, S1, n, p1, false, false);
  if (gt1) axis_pass(V2, A1, n, n, 1, 0, D1, n, p1, false, false);
  if (gd) axis_pass(N2, B0, n, n, 1, 0, S1, n, p1, false, false);
  __syncthreads();
  if (val) axis_pass(A0, val, p1, n, 1, 1, S2, n, p2, false, false);
  if (gt2) axis_pass(A0, gt2, p1, n, 1, 1, D2, n, p2, false, false);
  if (gt1) axis_pass(A1, gt1, p1, n, 1, 1, S2, n, p2, false, false);
  if (gd) axis_pass(B0, gd, p1, n, 1, 1, S2, n, p2, false, false);
  __syncthreads();
}

// r (n^3) += face integral of [ f phi + hd dphi/dxi_d + ht1 dphi/dxi_t1 + ht2 dphi/dxi_t2 ] at the
// face points (inputs may be null).
template <typename T>
__device__ void integrate_face(const T *f, const T *hd, const T *ht1, const T *ht2, int n, int d, int side,
                               const T *dend, const T *S1, const T *D1, int p1, const T *S2, const T *D2, int p2,
                               T *r, T *tmp) {
  int t1, t2;
  face_axes(d, t1, t2);
  const int nn = n * n;
  const int sz = n * max(n, p1);
  T *C0 = tmp, *C1 = tmp + sz, *C2 = tmp + 2 * sz, *F2 = tmp + 3 * sz, *G2 = tmp + 3 * sz + nn;
  bool c0 = false;
  if (f) { axis_pass(f, C0, p1, p2, 1, 1, S2, n, p2, true, false); c0 = true; }
  if (ht2) { axis_pass(ht2, C0, p1, p2, 1, 1, D2, n, p2, true, c0); c0 = true; }
  if (ht1) axis_pass(ht1, C1, p1, p2, 1, 1, S2, n, p2, true, false);
  if (hd) axis_pass(hd, C2, p1, p2, 1, 1, S2, n, p2, true, false);
  __syncthreads();
  bool f2 = false;
  if (c0) { axis_pass(C0, F2, p1, n, 1, 0, S1, n, p1, true, false); f2 = true; }
  if (ht1) { axis_pass(C1, F2, p1, n, 1, 0, D1, n, p1, true, f2); f2 = true; }
  if (hd) axis_pass(C2, G2, p1, n, 1, 0, S1, n, p1, true, false);
  __syncthreads();
  const int layer = side ? n - 1 : 0;
  for (int t = threadIdx.x; t < nn; t += blockDim.x) {
    const int i1 = t % n, i2 = t / n;
    if (f2) r[node_index(d, t1, t2, layer, i1, i2, n)] += F2[t];
    if (hd) {
      const T g = G2[t];
      for (int j = 0; j < n; ++j) r[node_index(d, t1, t2, j, i1, i2, n)] += dend[j] * g;
    }
  }
  __syncthreads();
}

// Deterministic block reduction of nout outputs, each a sum over npts of vals(o, p), added to
// out[o]. One warp per output (round-robin), lanes stride the points, shuffle tree at the end.
template <typename T, typename F>
__device__ void reduce_outputs(int nout, int npts, F vals, T *out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = warp; o < nout; o += nw) {
    T s = T(0);
    for (int p = lane; p < npts; p += 32) s += vals(o, p);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) out[o] += s;
  }
  __syncthreads();
}

// Trilinear Q1 weights N_v and reference gradients at a reference point.
template <typename T>
__device__ __forceinline__ void q1_weights(const T xi[3], T N[8], T dN[8][3]) {
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    T f[3], df[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int b = (v >> d) & 1;
      f[d] = b ? xi[d] : T(1) - xi[d];
      df[d] = b ? T(1) : T(-1);
    }
    N[v] = f[0] * f[1] * f[2];
    dN[v][0] = df[0] * f[1] * f[2];
    dN[v][1] = f[0] * df[1] * f[2];
    dN[v][2] = f[0] * f[1] * df[2];
  }
}

// Enrichment of one component at a point with 1-D weight factors f: sN = sum_v N_v e_v and
// sD_d = sum_v dN_v/dxi_d e_v over the 8 trilinear weights (e: 8 coefficients); with the constant
// weight (l = 0) sN = e_0 and sD = 0.
template <typename T, bool GRADN>
__device__ __forceinline__ void enr_trial(const T f[3][2], const T *e, bool l0, T &sN, T sD[3]) {
  sN = T(0);
  sD[0] = sD[1] = sD[2] = T(0);
  if (l0) {
    sN = e[0];
    return;
  }
  // nested linear interpolation, x then y then z (FP64 operations are the scarce resource of this
  // kernel): the value, and each derivative as the difference along its axis interpolated along the
  // other two; cx/dx per (b1, b2), j = b1 + 2 b2
  T cx[4], dx[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const T e0 = e[2 * j], e1 = e[2 * j + 1];
    cx[j] = f[0][0] * e0 + f[0][1] * e1;
    dx[j] = e1 - e0;
  }
  T cy[2], dy[2], dxy[2];
#pragma unroll
  for (int b2 = 0; b2 < 2; ++b2) {
    cy[b2] = f[1][0] * cx[2 * b2] + f[1][1] * cx[2 * b2 + 1];
    dy[b2] = cx[2 * b2 + 1] - cx[2 * b2];
    dxy[b2] = f[1][0] * dx[2 * b2] + f[1][1] * dx[2 * b2 + 1];
  }
  sN = f[2][0] * cy[0] + f[2][1] * cy[1];
  if (GRADN) {
    sD[0] = f[2][0] * dxy[0] + f[2][1] * dxy[1];
    sD[1] = f[2][0] * dy[0] + f[2][1] * dy[1];
    sD[2] = cy[1] - cy[0];
  }
}

// acc[a * 8 + v] += beta_a N_v + sum_e alpha_a[e] dN_v/dxi_e over the 8 trilinear weights at a point
// with 1-D factors f. With N_v = F0 F1 F2 (F_e = f[e][b_e]) and dN_v/dxi_e = s_e (product of the
// other two), s_e = +1 for b_e = 1 and -1 for b_e = 0, the term is
// F1 F2 (beta F0 + s0 alpha_0) + F0 (s1 alpha_1 F2 + s2 alpha_2 F1).
template <typename T>
__device__ __forceinline__ void acc_trilinear(const T f[3][2], const T beta[3], const T alpha[3][3], T *acc) {
  T F12[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) F12[j] = f[1][j & 1] * f[2][j >> 1];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T P0 = beta[a] * f[0][0] - alpha[a][0], P1 = beta[a] * f[0][1] + alpha[a][0];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b1 = j & 1, b2 = j >> 1;
      const T Q = (b1 ? alpha[a][1] : -alpha[a][1]) * f[2][b2] + (b2 ? alpha[a][2] : -alpha[a][2]) * f[1][b1];
      acc[a * 8 + 2 * j] += F12[j] * P0 + f[0][0] * Q;
      acc[a * 8 + 2 * j + 1] += F12[j] * P1 + f[0][1] * Q;
    }
  }
}

}  // namespace dgw
