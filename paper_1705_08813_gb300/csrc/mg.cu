// Geometric multigrid preconditioner for the pressure Poisson problem (the paper solves it with
// a matrix-free multigrid-preconditioned CG, Sec. 4.4; its multigrid details are not given, so
// this design is our own): h-coarsening of the tanh-graded channel by factors of two, first in
// the wall-normal direction alone while the wall cells are thin, then in every direction whose
// cell count is even (coarse vertex rows are every other fine row, so the meshes nest), the same
// degree k on every level, re-discretised SIPG level operators,
// Chebyshev smoothing with the inverse diagonal, DG embedding (prolongation) and its transpose
// (restriction). The coarsest level is solved with a dense (A + c 1 1^T)^-1 computed on the device,
// either at degree k (when its n_p <= 2400) or after one more level with Q_1 on the same cells
// (when 8 x cells <= 2400); only a hierarchy too large for both falls back to a fixed number of
// device-side Jacobi-PCG steps there.
// Mode 1 runs the whole V-cycle in FP32 (operators, smoothers, transfers) on a residual scaled
// by its RMS value; mode 0 runs it in FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "solver.h"
#include "sumfac.cuh"

namespace dgw {

constexpr double kSmoothRange = 45.0;   // Chebyshev smooths [1.1 lmax/45, 1.1 lmax]
constexpr double kLmaxSafety = 1.1;     // on the CG-Lanczos estimate, which approaches lmax from below
constexpr int kCoarseIters = 24;       // PCG steps on the coarsest level
constexpr int kLanczos = 24;           // CG-Lanczos steps for lmax(D^-1 A)
constexpr double kSemiRatio = 0.5;      // y-only coarsening while 2 min h_y <= this x min(h_x, h_z)
constexpr long kDenseMax = 2400;       // coarsest systems up to this size are solved densely (the
                                       // hierarchy stops coarsening once Q_1 on its cells fits)

// ------------------------------------------------------------------------------------------
// vector kernels (templated on the level precision; reductions accumulate in double)
// ------------------------------------------------------------------------------------------

// column blockIdx.y of a block of vectors (n values each); partial sums per column
template <typename T>
__global__ void mg_dot_partial(const T *__restrict__ a, const T *__restrict__ b, long n, double *__restrict__ partial) {
  a += (size_t)blockIdx.y * n;
  if (b) b += (size_t)blockIdx.y * n;
  partial += (size_t)blockIdx.y * gridDim.x;
  double s = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    s += b ? (double)a[i] * (double)b[i] : (double)a[i];
  __shared__ double wp[32];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) wp[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? wp[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

// one warp per column (blockIdx.x); the column's scalars are out[column * MS_COUNT + slot]
__global__ void mg_dot_finish(const double *__restrict__ partial, int np, double *out, int slot) {
  partial += (size_t)blockIdx.x * np;
  out += (size_t)blockIdx.x * 8;
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += 32) s += partial[i];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (threadIdx.x == 0) out[slot] = s;
}

constexpr int MG_RED = 152;

// per column c < ncols: sc[c * MS_COUNT + slot] = sum_i a_ci b_ci (b null: sum_i a_ci)
template <typename T>
static void mg_reduce(const T *a, const T *b, long n, double *partial, double *sc, int slot, cudaStream_t s,
                      int ncols = 1) {
  note_launch();
  mg_dot_partial<T><<<dim3(MG_RED, ncols), 256, 0, s>>>(a, b, n, partial);
  note_launch();
  mg_dot_finish<<<ncols, 32, 0, s>>>(partial, MG_RED, sc, slot);
}

static inline int mg_grid(long n) {
  long g = (n + 255) / 256;
  return (int)std::min<long>(std::max<long>(g, 1), 152 * 8);
}

// slots of the level scalars (MS_COUNT per column; mg_dot_finish strides columns by 8)
enum { MS_RZ = 0, MS_RZNEW, MS_DQ, MS_SUM, MS_COUNT = 8 };
static_assert(MS_COUNT == 8, "mg_dot_finish column stride");

// Chebyshev step: r = b - t (t = A x); d = c1 d + c2 D^-1 r; x += d (first: d = c2 D^-1 r)
template <typename T>
__global__ void cheb_step(T *__restrict__ x, T *__restrict__ d, const T *__restrict__ b, const T *__restrict__ t,
                          const T *__restrict__ dinv, long n, T c1, T c2, int first, int zero_x) {
  const size_t co = (size_t)blockIdx.y * n;   // column of a block of vectors (dinv shared)
  x += co; d += co; b += co; t += co;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const T r = zero_x ? b[i] : b[i] - t[i];
    const T dn = (first ? T(0) : c1 * d[i]) + c2 * dinv[i] * r;
    d[i] = dn;
    x[i] = (zero_x ? T(0) : x[i]) + dn;
  }
}

template <typename T>
__global__ void residual_kernel(T *__restrict__ r, const T *__restrict__ b, const T *__restrict__ t, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) r[i] = b[i] - t[i];
}

// coarse PCG pieces (scalars on the device)
template <typename T>
__global__ void cpcg_update(T *__restrict__ x, T *__restrict__ r, const T *__restrict__ d, const T *__restrict__ t,
                            long n, const double *sc) {
  const double alpha = sc[MS_DQ] != 0.0 ? sc[MS_RZ] / sc[MS_DQ] : 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    x[i] = (T)((double)x[i] + alpha * (double)d[i]);
    r[i] = (T)((double)r[i] - alpha * (double)t[i]);
  }
}

template <typename T>
__global__ void cpcg_precond(T *__restrict__ z, const T *__restrict__ r, const T *__restrict__ dinv, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) z[i] = dinv[i] * r[i];
}

template <typename T>
__global__ void sub_mean_T(T *__restrict__ z, long n, const double *sc, int slot) {
  z += (size_t)blockIdx.y * n;
  const double m = sc[(size_t)blockIdx.y * MS_COUNT + slot] / (double)n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    z[i] = (T)((double)z[i] - m);
}

template <typename T>
__global__ void cpcg_direction(T *__restrict__ d, const T *__restrict__ z, long n, double *sc, int first) {
  const double beta = (first || sc[MS_RZ] == 0.0) ? 0.0 : sc[MS_RZNEW] / sc[MS_RZ];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    d[i] = first ? z[i] : (T)((double)z[i] + beta * (double)d[i]);   // d unread on the first step
}

__global__ void shift_scalar(double *sc, int dst, int src) {
  if (threadIdx.x == 0) sc[dst] = sc[src];
}

// FP64 residual -> level-0 right-hand side scaled by 1/rms(r); rms from the CG scalar RR.
template <typename T>
__global__ void scale_in(T *__restrict__ b0, const double *__restrict__ r, long n, const double *csc, int rr_slot) {
  const double rr = csc[rr_slot];
  const double s = rr > 0.0 ? sqrt((double)n / rr) : 1.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    b0[i] = (T)(r[i] * s);
}
template <typename T>
__global__ void scale_out(double *__restrict__ z, const T *__restrict__ x0, long n, const double *csc, int rr_slot) {
  const double rr = csc[rr_slot];
  const double s = rr > 0.0 ? sqrt(rr / (double)n) : 1.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    z[i] = (double)x0[i] * s;
}

template <typename T>
__global__ void inv_kernel(const double *__restrict__ dg, T *__restrict__ dinv, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    dinv[i] = (T)(1.0 / dg[i]);
}

template <typename T>
__global__ void scale_vec(T *__restrict__ y, const T *__restrict__ x, long n, const double *sc, int slot) {
  const double nrm = sqrt(sc[slot]);
  const double s = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = (T)((double)x[i] * s);
}

template <typename T>
__global__ void mul_kernel(T *__restrict__ y, const T *__restrict__ a, const T *__restrict__ b, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) y[i] = a[i] * b[i];
}

// ------------------------------------------------------------------------------------------
// transfers: DG embedding of a coarse cell's polynomial into its children and the transpose
// ------------------------------------------------------------------------------------------

struct XferDims {
  int fnx, fny, fnz;   // fine cells
  int cnx, cny, cnz;   // coarse cells
  int cf[3];           // factors (1 or 2)
  const void *py;      // [cny][2][n*n] y-embeddings (graded rows split unevenly), when cf[1] == 2
};

// Transfers with one CTA per coarse cell and all its children: the 1-D passes are shared
// between the children (2n^4 + 4n^4 + 8n^4 FMAs for 8 children instead of 24n^4), every thread owns
// whole lines, and n is a compile-time constant. Directions that are not coarsened (cf = 1) use the
// identity.
template <typename T, int K>
__device__ __forceinline__ void load_xfer_matrices(const Basis<T> &B, const XferDims &X, int cj, T (*Pm)[2][(K + 1) * (K + 1)]) {
  constexpr int n = K + 1, n2 = n * n;
  const T *py = static_cast<const T *>(X.py);
  for (int t = threadIdx.x; t < 3 * 2 * n2; t += blockDim.x) {
    const int d = t / (2 * n2), o = (t / n2) % 2, e = t % n2;
    T v = (e / n == e % n) ? T(1) : T(0);
    if (X.cf[d] == 2) v = d == 1 ? py[((size_t)cj * 2 + o) * n2 + e] : B.P[o][e];
    Pm[d][o][e] = v;
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(256) prolong_cell_kernel(const Basis<T> *Bg, XferDims X, const T *__restrict__ xc,
                                                           T *__restrict__ xf) {
  constexpr int n = K + 1, n2 = n * n, n3 = n2 * n;
  __shared__ T Pm[3][2][n2];
  __shared__ T Xc[n3], A[2 * n3], Bm[4 * n3];
  const int cc = blockIdx.x;
  xc += (size_t)blockIdx.y * gridDim.x * n3;   // column of a block of vectors
  xf += (size_t)blockIdx.y * X.fnx * X.fny * X.fnz * n3;
  const int ci = cc % X.cnx, cj = (cc / X.cnx) % X.cny, ck = cc / (X.cnx * X.cny);
  const int c0 = X.cf[0], c1 = X.cf[1], c2 = X.cf[2];
  load_xfer_matrices<T, K>(*Bg, X, cj, Pm);
  for (int t = threadIdx.x; t < n3; t += blockDim.x) Xc[t] = xc[(size_t)cc * n3 + t];
  __syncthreads();
  for (int it = threadIdx.x; it < c0 * n2; it += blockDim.x) {   // x: (ox, line y,z)
    const int ox = it / n2, l = it - ox * n2;
    T v[n];
#pragma unroll
    for (int b = 0; b < n; ++b) v[b] = Xc[n * l + b];
#pragma unroll
    for (int a = 0; a < n; ++a) {
      T s = T(0);
#pragma unroll
      for (int b = 0; b < n; ++b) s += Pm[0][ox][a * n + b] * v[b];
      A[ox * n3 + n * l + a] = s;
    }
  }
  __syncthreads();
  for (int it = threadIdx.x; it < c0 * c1 * n2; it += blockDim.x) {   // y: (ox, oy, line x,z)
    const int o = it / n2, l = it - o * n2, ox = o % c0, oy = o / c0;
    const int x = l % n, z = l / n;
    T v[n];
#pragma unroll
    for (int b = 0; b < n; ++b) v[b] = A[ox * n3 + x + n * b + n2 * z];
#pragma unroll
    for (int a = 0; a < n; ++a) {
      T s = T(0);
#pragma unroll
      for (int b = 0; b < n; ++b) s += Pm[1][oy][a * n + b] * v[b];
      Bm[(ox * 2 + oy) * n3 + x + n * a + n2 * z] = s;
    }
  }
  __syncthreads();
  for (int it = threadIdx.x; it < c0 * c1 * c2 * n2; it += blockDim.x) {   // z: (ox, oy, oz, line x,y)
    const int o = it / n2, l = it - o * n2, ox = o % c0, oy = (o / c0) % c1, oz = o / (c0 * c1);
    const int fc = (ci * c0 + ox) + X.fnx * ((cj * c1 + oy) + X.fny * (ck * c2 + oz));
    T v[n];
#pragma unroll
    for (int b = 0; b < n; ++b) v[b] = Bm[(ox * 2 + oy) * n3 + l + n2 * b];
    T *out = xf + (size_t)fc * n3 + l;
#pragma unroll
    for (int a = 0; a < n; ++a) {
      T s = T(0);
#pragma unroll
      for (int b = 0; b < n; ++b) s += Pm[2][oz][a * n + b] * v[b];
      out[n2 * a] += s;
    }
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(256) restrict_cell_kernel(const Basis<T> *Bg, XferDims X, const T *__restrict__ rf,
                                                            T *__restrict__ rc) {
  constexpr int n = K + 1, n2 = n * n, n3 = n2 * n;
  __shared__ T Pm[3][2][n2];
  __shared__ T Rf[8 * n3], Zs[4 * n3], Ys[2 * n3];
  const int cc = blockIdx.x;
  rc += (size_t)blockIdx.y * gridDim.x * n3;   // column of a block of vectors
  rf += (size_t)blockIdx.y * X.fnx * X.fny * X.fnz * n3;
  const int ci = cc % X.cnx, cj = (cc / X.cnx) % X.cny, ck = cc / (X.cnx * X.cny);
  const int c0 = X.cf[0], c1 = X.cf[1], c2 = X.cf[2];
  load_xfer_matrices<T, K>(*Bg, X, cj, Pm);
  const int nch = c0 * c1 * c2;
  for (int t = threadIdx.x; t < nch * n3; t += blockDim.x) {
    const int o = t / n3, e = t - o * n3, ox = o % c0, oy = (o / c0) % c1, oz = o / (c0 * c1);
    const int fc = (ci * c0 + ox) + X.fnx * ((cj * c1 + oy) + X.fny * (ck * c2 + oz));
    Rf[((ox * 2 + oy) * 2 + oz) * n3 + e] = rf[(size_t)fc * n3 + e];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < c0 * c1 * n2; it += blockDim.x) {   // z (summed over oz): (ox, oy, line x,y)
    const int o = it / n2, l = it - o * n2, ox = o % c0, oy = o / c0;
    T acc[n];
#pragma unroll
    for (int a = 0; a < n; ++a) acc[a] = T(0);
    for (int oz = 0; oz < c2; ++oz) {
      T v[n];
#pragma unroll
      for (int b = 0; b < n; ++b) v[b] = Rf[((ox * 2 + oy) * 2 + oz) * n3 + l + n2 * b];
#pragma unroll
      for (int a = 0; a < n; ++a)
#pragma unroll
        for (int b = 0; b < n; ++b) acc[a] += Pm[2][oz][b * n + a] * v[b];
    }
#pragma unroll
    for (int a = 0; a < n; ++a) Zs[(ox * 2 + oy) * n3 + l + n2 * a] = acc[a];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < c0 * n2; it += blockDim.x) {   // y (summed over oy): (ox, line x,z)
    const int ox = it / n2, l = it - ox * n2, x = l % n, z = l / n;
    T acc[n];
#pragma unroll
    for (int a = 0; a < n; ++a) acc[a] = T(0);
    for (int oy = 0; oy < c1; ++oy) {
      T v[n];
#pragma unroll
      for (int b = 0; b < n; ++b) v[b] = Zs[(ox * 2 + oy) * n3 + x + n * b + n2 * z];
#pragma unroll
      for (int a = 0; a < n; ++a)
#pragma unroll
        for (int b = 0; b < n; ++b) acc[a] += Pm[1][oy][b * n + a] * v[b];
    }
#pragma unroll
    for (int a = 0; a < n; ++a) Ys[ox * n3 + x + n * a + n2 * z] = acc[a];
  }
  __syncthreads();
  for (int l = threadIdx.x; l < n2; l += blockDim.x) {   // x (summed over ox): line y,z
    T acc[n];
#pragma unroll
    for (int a = 0; a < n; ++a) acc[a] = T(0);
    for (int ox = 0; ox < c0; ++ox) {
      T v[n];
#pragma unroll
      for (int b = 0; b < n; ++b) v[b] = Ys[ox * n3 + n * l + b];
#pragma unroll
      for (int a = 0; a < n; ++a)
#pragma unroll
        for (int b = 0; b < n; ++b) acc[a] += Pm[0][ox][b * n + a] * v[b];
    }
#pragma unroll
    for (int a = 0; a < n; ++a) rc[(size_t)cc * n3 + n * l + a] = acc[a];
  }
}

template <typename T>
static void launch_restrict(const Basis<T> *B, const XferDims &X, int n, const T *rf, T *rc, int ncoarse,
                            cudaStream_t s, int ncols = 1) {
  note_launch();
  const dim3 g(ncoarse, ncols);
  switch (n) {
    case 2: restrict_cell_kernel<T, 1><<<g, 128, 0, s>>>(B, X, rf, rc); break;
    case 3: restrict_cell_kernel<T, 2><<<g, 128, 0, s>>>(B, X, rf, rc); break;
    case 4: restrict_cell_kernel<T, 3><<<g, 128, 0, s>>>(B, X, rf, rc); break;
    case 5: restrict_cell_kernel<T, 4><<<g, 128, 0, s>>>(B, X, rf, rc); break;
    default: restrict_cell_kernel<T, 5><<<g, 160, 0, s>>>(B, X, rf, rc); break;
  }
}

template <typename T>
static void launch_prolong(const Basis<T> *B, const XferDims &X, int n, const T *xc, T *xf, int ncoarse,
                           cudaStream_t s, int ncols = 1) {
  note_launch();
  const dim3 g(ncoarse, ncols);
  switch (n) {
    case 2: prolong_cell_kernel<T, 1><<<g, 64, 0, s>>>(B, X, xc, xf); break;
    case 3: prolong_cell_kernel<T, 2><<<g, 96, 0, s>>>(B, X, xc, xf); break;
    case 4: prolong_cell_kernel<T, 3><<<g, 128, 0, s>>>(B, X, xc, xf); break;
    case 5: prolong_cell_kernel<T, 4><<<g, 224, 0, s>>>(B, X, xc, xf); break;
    default: prolong_cell_kernel<T, 5><<<g, 256, 0, s>>>(B, X, xc, xf); break;
  }
}

// p-transfer between Q_k and Q_1 on the same cells: P1[i*2 + j] = linear Lagrange j at the
// Gauss-Lobatto node z_i of degree k (prolongation: nodal interpolation, restriction: transpose).
template <typename T>
__global__ void p_prolongate_add(const T *__restrict__ P1, int n, const T *__restrict__ x1, T *__restrict__ xk) {
  __shared__ T A[NMAX * NMAX * NMAX], Bv[NMAX * NMAX * NMAX], Pm[NMAX * 2];
  const int c = blockIdx.x, n3 = n * n * n;
  x1 += (size_t)blockIdx.y * gridDim.x * 8;    // column of a block of vectors
  xk += (size_t)blockIdx.y * gridDim.x * n3;
  for (int t = threadIdx.x; t < 2 * n; t += blockDim.x) Pm[t] = P1[t];
  for (int t = threadIdx.x; t < 8; t += blockDim.x) A[t] = x1[(size_t)c * 8 + t];
  __syncthreads();
  axis_pass(A, Bv, 2, 2, 2, 0, Pm, 2, n, false, false);
  __syncthreads();
  axis_pass(Bv, A, n, 2, 2, 1, Pm, 2, n, false, false);
  __syncthreads();
  axis_pass(A, Bv, n, n, 2, 2, Pm, 2, n, false, false);
  __syncthreads();
  for (int t = threadIdx.x; t < n3; t += blockDim.x) xk[(size_t)c * n3 + t] += Bv[t];
}

template <typename T>
__global__ void p_restrict(const T *__restrict__ P1, int n, const T *__restrict__ rk, T *__restrict__ r1) {
  __shared__ T A[NMAX * NMAX * NMAX], Bv[NMAX * NMAX * NMAX], Pm[NMAX * 2];
  const int c = blockIdx.x, n3 = n * n * n;
  rk += (size_t)blockIdx.y * gridDim.x * n3;   // column of a block of vectors
  r1 += (size_t)blockIdx.y * gridDim.x * 8;
  for (int t = threadIdx.x; t < 2 * n; t += blockDim.x) Pm[t] = P1[t];
  for (int t = threadIdx.x; t < n3; t += blockDim.x) A[t] = rk[(size_t)c * n3 + t];
  __syncthreads();
  axis_pass(A, Bv, n, n, n, 0, Pm, 2, n, true, false);
  __syncthreads();
  axis_pass(Bv, A, 2, n, n, 1, Pm, 2, n, true, false);
  __syncthreads();
  axis_pass(A, Bv, 2, 2, n, 2, Pm, 2, n, true, false);
  __syncthreads();
  for (int t = threadIdx.x; t < 8; t += blockDim.x) r1[(size_t)c * 8 + t] = Bv[t];
}

// x = Ainv b (one warp per row, lanes stride the row)
template <typename T>
__global__ void dense_gemv(const T *__restrict__ Ainv, const T *__restrict__ b, T *__restrict__ x, int N) {
  b += (size_t)blockIdx.y * N;   // column of a block of vectors
  x += (size_t)blockIdx.y * N;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= N) return;
  const T *row = Ainv + (size_t)warp * N;
  double s = 0.0;
  for (int j = lane; j < N; j += 32) s += (double)row[j] * (double)b[j];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) x[warp] = (T)s;
}


// ------------------------------------------------------------------------------------------
// hierarchy
// ------------------------------------------------------------------------------------------

template <typename T>
struct Lvl {
  BoxGeometry geo;
  MeshView<T> view;
  long n = 0;
  T *dinv = nullptr, *x = nullptr, *b = nullptr, *r = nullptr, *d = nullptr, *t = nullptr, *z = nullptr;
  T *x2 = nullptr;   // second iterate buffer of the fused Chebyshev steps
  double *sc = nullptr, *partial = nullptr;
  double lmax = 1.0;
  XferDims to_coarse{};   // transfer to the next coarser level
  const T *p1 = nullptr;  // when set: the next level is Q_1 on the same cells (p-transfer table)
  const T *ainv = nullptr; // coarsest level solved densely with this inverse (N = n)
  std::vector<void *> allocs;
};

// cols: columns every level vector holds (a block of right-hand sides); ncols: columns one V-cycle
// processes (<= cols)
template <typename T>
struct Hierarchy {
  std::vector<Lvl<T> *> L;
  int cheb = 5;
  const Basis<T> *basis = nullptr;
  int cols = 1, ncols = 1;
};

}  // namespace dgw

struct dgw::MGLevel {
  int prec = -1;   // 0 double, 1 float
  void *h = nullptr;
};

namespace dgw {

// Allocation zeroed on the solver stream (all multigrid work runs on that non-blocking stream; a
// plain cudaMemset would run on the legacy stream and could race with it).
template <typename T>
static T *lalloc(Lvl<T> *L, size_t n, cudaError_t &e, cudaStream_t s) {
  void *p = nullptr;
  if (e != cudaSuccess) return nullptr;
  e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
  if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, std::max<size_t>(n, 1) * sizeof(T), s);
  if (e == cudaSuccess) L->allocs.push_back(p);
  return (T *)p;
}

// Gauss-Jordan inversion in place on the device (FP64, no pivoting: the matrices inverted here are
// symmetric positive definite, whose pivots stay positive). Step k saves the scaled pivot row R and
// the pivot column C, then updates every entry: A_ij -= C_i R_j (A_ik -> -C_i / p, row k -> R).
__global__ void gj_pivot_kernel(const double *__restrict__ A, int N, int k, double *__restrict__ R,
                                double *__restrict__ Cc) {
  const double p = A[(size_t)k * N + k];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    R[j] = j == k ? 1.0 / p : A[(size_t)k * N + j] / p;
    Cc[j] = A[(size_t)j * N + k];
  }
}

__global__ void gj_update_kernel(double *__restrict__ A, int N, int k, const double *__restrict__ R,
                                 const double *__restrict__ Cc) {
  const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double *a = A + (size_t)i * N + j;
  if (i == k) *a = R[j];
  else *a = (j == k ? 0.0 : *a) - Cc[i] * R[j];
}

template <typename T>
__global__ void narrow_kernel(const double *__restrict__ a, T *__restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (T)a[i];
}

// Inverse of A + c 1 1^T (SPD when the null space of A is the constants; on zero-mean right-hand
// sides it acts as the pseudo-inverse of A and returns zero-mean solutions), c 1 1^T adding
// trace(A)/N^2 to every entry. Computed on the device into out (N x N, type T, allocated on the
// level). Returns false, leaving out unset, if the inverse has a non-positive or non-finite
// diagonal entry (the caller keeps the iterative coarse solve).
template <typename T>
static bool dense_inverse_device(Lvl<T> *D, std::vector<double> A, int N, T **out, cudaError_t &e, cudaStream_t s) {
  double tr = 0.0;
  for (int i = 0; i < N; ++i) tr += A[(size_t)i * N + i];
  const double c = tr / N;
  for (size_t i = 0; i < (size_t)N * N; ++i) A[i] += c / N;
  double *Ad = nullptr, *R = nullptr, *Cc = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&Ad, (size_t)N * N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&R, (size_t)N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&Cc, (size_t)N * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(Ad, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // A's staging copy may go now
  const dim3 ug((N + 255) / 256, N);
  for (int k = 0; k < N && e == cudaSuccess; ++k) {
    gj_pivot_kernel<<<(N + 255) / 256, 256, 0, s>>>(Ad, N, k, R, Cc);
    gj_update_kernel<<<ug, 256, 0, s>>>(Ad, N, k, R, Cc);
    if ((k & 255) == 255) e = cudaGetLastError();
  }
  note_launches(2ull * N);
  bool ok = false;
  if (e == cudaSuccess) {
    std::vector<double> diag(N);
    for (int i = 0; i < N && e == cudaSuccess; ++i)   // the inverse's diagonal must be positive and finite
      e = cudaMemcpyAsync(&diag[i], Ad + (size_t)i * N + i, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    ok = e == cudaSuccess;
    for (int i = 0; i < N && ok; ++i) ok = std::isfinite(diag[i]) && diag[i] > 0.0;
  }
  if (ok) {
    T *o = lalloc<T>(D, (size_t)N * N, e, s);
    if (e == cudaSuccess) {
      note_launch();
      narrow_kernel<T><<<1216, 256, 0, s>>>(Ad, o, (size_t)N * N);
      e = cudaStreamSynchronize(s);
    }
    if (e == cudaSuccess) *out = o;
    else ok = false;
  }
  if (Ad) cudaFree(Ad);
  if (R) cudaFree(R);
  if (Cc) cudaFree(Cc);
  return ok;
}

template <typename T>
static void free_hier(Hierarchy<T> *H) {
  if (!H) return;
  for (auto *L : H->L) {
    for (void *p : L->allocs) cudaFree(p);
    delete L;
  }
  delete H;
}

template <typename T>
static cudaError_t level_apply(const Lvl<T> *L, const T *x, T *y, cudaStream_t s) {
  return launch_laplace<T>(L->view, x, y, s);
}

// Largest eigenvalue of D^-1 A from the Lanczos tridiagonal of kLanczos Jacobi-PCG steps on a
// random zero-mean right-hand side (setup only; host-synchronising). The Ritz value approaches
// lmax from below; the smoother applies the safety factor kLmaxSafety.
static double tridiag_max_eig(const std::vector<double> &a, const std::vector<double> &b) {
  // Sturm-sequence bisection for the largest eigenvalue of the symmetric tridiagonal (a, b)
  const int m = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {   // eigenvalues < x
    int c = 0;
    double q = a[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < m; ++i) {
      if (q == 0.0) q = 1e-300;
      q = a[i] - x - b[i - 1] * b[i - 1] / q;
      if (q < 0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) < m) lo = mid; else hi = mid;
  }
  return hi;
}

template <typename T>
static cudaError_t estimate_lmax(Lvl<T> *L, cudaStream_t s) {
  const long n = L->n;
  const int G = mg_grid(n);
  std::vector<T> h(n);
  uint64_t st = 0x243F6A8885A308D3ull;
  for (long i = 0; i < n; ++i) {
    st ^= st << 13; st ^= st >> 7; st ^= st << 17;
    h[i] = (T)((double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5);
  }
  cudaError_t e = cudaMemcpyAsync(L->r, h.data(), n * sizeof(T), cudaMemcpyHostToDevice, s);
  // r zero-mean; z = D^-1 r (zero-mean); d = z
  mg_reduce<T>(L->r, nullptr, n, L->partial, L->sc, MS_SUM, s);
  sub_mean_T<T><<<G, 256, 0, s>>>(L->r, n, L->sc, MS_SUM);
  std::vector<double> alpha, beta;
  double host[MS_COUNT];
  double rz_old = 0.0;
  for (int it = 0; it < kLanczos && e == cudaSuccess; ++it) {
    cpcg_precond<T><<<G, 256, 0, s>>>(L->z, L->r, L->dinv, n);
    mg_reduce<T>(L->z, nullptr, n, L->partial, L->sc, MS_SUM, s);
    sub_mean_T<T><<<G, 256, 0, s>>>(L->z, n, L->sc, MS_SUM);
    mg_reduce<T>(L->r, L->z, n, L->partial, L->sc, MS_RZNEW, s);
    cpcg_direction<T><<<G, 256, 0, s>>>(L->d, L->z, n, L->sc, it == 0);
    shift_scalar<<<1, 32, 0, s>>>(L->sc, MS_RZ, MS_RZNEW);
    e = level_apply(L, L->d, L->t, s);
    mg_reduce<T>(L->d, L->t, n, L->partial, L->sc, MS_DQ, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, L->sc, sizeof(host), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    const double rz = host[MS_RZ], dq = host[MS_DQ];
    if (!(rz > 0.0) || !(dq > 0.0)) break;
    if (it > 0) beta.push_back(rz / rz_old);
    alpha.push_back(rz / dq);
    rz_old = rz;
    cpcg_update<T><<<G, 256, 0, s>>>(L->x, L->r, L->d, L->t, n, L->sc);
  }
  if (e != cudaSuccess || alpha.empty()) return e;
  // Lanczos tridiagonal from the CG coefficients
  const int m = (int)alpha.size();
  std::vector<double> ta(m), tb(std::max(m - 1, 0));
  for (int i = 0; i < m; ++i) {
    ta[i] = 1.0 / alpha[i] + (i > 0 ? beta[i - 1] / alpha[i - 1] : 0.0);
    if (i + 1 < m) tb[i] = std::sqrt(beta[i]) / alpha[i];
  }
  L->lmax = tridiag_max_eig(ta, tb);
  return cudaSuccess;
}

// Curved levels: metric tables of a coarser mesh over the same map, uploaded in precision X.
template <typename X>
static void upload_curved(Lvl<X> *L, const CurvedHost &g, MeshView<X> &v, cudaError_t &e, cudaStream_t s) {
  auto up = [&](const std::vector<double> &h) -> const X * {
    std::vector<X> hx(h.begin(), h.end());
    X *d = lalloc<X>(L, hx.size(), e, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, hx.data(), hx.size() * sizeof(X), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the staging vector dies here
    return d;
  };
  v.geo = GEO_CURVED;
  // the pressure levels carry no enrichment: the tables of the default point sets only
  for (int t = 0; t < NMVOL; ++t) v.mvol[t] = g.mvol[t].empty() ? nullptr : up(g.mvol[t]);
  for (int t = 0; t < NQSET; ++t) v.mxf[t] = up(g.mxf[t]);
  for (int t = 0; t < NQSET; ++t) v.myf[t] = g.myf[t].empty() ? nullptr : up(g.myf[t]);
  v.lvol = up(g.lvol);
  v.lface = up(g.lface);
  std::vector<double> tau((size_t)g.nx * g.ny * g.nz);
  for (size_t c = 0; c < tau.size(); ++c) tau[c] = g.tau[c % ((size_t)g.nx * g.ny)];
  v.tau = up(tau);
  v.hy = nullptr;
  v.rowops = nullptr;
}

// Dense matrix of a level operator, assembled on the device column by column from the FP64
// operator of the level (curved meshes have no host-side operator).
static cudaError_t assemble_device(const MeshView<double> &v, int N, std::vector<double> &A, cudaStream_t s) {
  double *I = nullptr, *Y = nullptr;
  cudaError_t e = cudaMalloc(&I, (size_t)N * N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&Y, (size_t)N * N * sizeof(double));
  std::vector<double> eye((size_t)N * N, 0.0);
  for (int j = 0; j < N; ++j) eye[(size_t)j * N + j] = 1.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(I, eye.data(), eye.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  for (int j = 0; j < N && e == cudaSuccess; ++j) e = launch_laplace<double>(v, I + (size_t)j * N, Y + (size_t)j * N, s);
  std::vector<double> cols((size_t)N * N);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cols.data(), Y, cols.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (I) cudaFree(I);
  if (Y) cudaFree(Y);
  A.assign((size_t)N * N, 0.0);
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) A[(size_t)i * N + j] = cols[(size_t)j * N + i];
  return e;
}

template <typename T>
static cudaError_t build_hierarchy(dgw_mesh *M, Hierarchy<T> *H, const MeshView<T> &fine, const T *fine_basis_dev,
                                   cudaStream_t s) {
  (void)fine_basis_dev;
  cudaError_t e = cudaSuccess;
  const bool curved = M->P.geometry == 1;
  const int k = M->P.degree, n = k + 1, n3 = n * n * n;
  int nx = M->P.nx, ny = M->P.ny, nz = M->P.nz;
  std::vector<double> yv = M->yv;
  MeshView<double> v64 = M->v64;   // FP64 view of the current level (curved: diagonal, dense assembly)
  for (int lev = 0; e == cudaSuccess; ++lev) {
    Lvl<T> *L = new Lvl<T>();
    H->L.push_back(L);
    box_geometry(k, nx, ny, nz, M->P.lx, M->P.lz, yv, L->geo);
    L->n = (long)nx * ny * nz * n3;
    if (lev == 0) {
      L->view = fine;
    } else {
      L->view = fine;
      L->view.nx = nx; L->view.ny = ny; L->view.nz = nz;
      L->view.nc = nx * ny * nz;
      L->view.ne = 0;
      L->view.np = L->n;
      L->view.hx = (T)L->geo.hx;
      L->view.hz = (T)L->geo.hz;
      L->view.enr = nullptr;
      L->view.slot = nullptr;
      if (curved) {
        CurvedHost cg;
        dgw_mesh_params Pl = M->P;
        Pl.full_quadrature = 0;   // no enriched cells on the pressure levels
        curved_geometry(Pl, nx, ny, nz, k, M->basis64, cg);
        upload_curved<T>(L, cg, L->view, e, s);
        v64 = M->v64;
        v64.nx = nx; v64.ny = ny; v64.nz = nz;
        v64.nc = nx * ny * nz;
        v64.ne = 0;
        v64.np = L->n;
        v64.enr = nullptr;
        v64.slot = nullptr;
        Lvl<double> tmp;   // owns nothing: the FP64 tables live with the level
        upload_curved<double>(&tmp, cg, v64, e, s);
        L->allocs.insert(L->allocs.end(), tmp.allocs.begin(), tmp.allocs.end());
      } else {
        std::vector<T> hy(L->geo.hy.begin(), L->geo.hy.end()), tau(L->geo.tau.begin(), L->geo.tau.end());
        T *hyd = lalloc<T>(L, hy.size(), e, s), *taud = lalloc<T>(L, tau.size(), e, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hyd, hy.data(), hy.size() * sizeof(T), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(taud, tau.data(), tau.size() * sizeof(T), cudaMemcpyHostToDevice, s);
        L->view.hy = hyd;
        L->view.tau = taud;
        std::vector<double> rops;
        box_rowscal(L->geo, rops);
        std::vector<T> ropsT(rops.begin(), rops.end());
        T *rd = lalloc<T>(L, ropsT.size(), e, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(rd, ropsT.data(), ropsT.size() * sizeof(T), cudaMemcpyHostToDevice, s);
        L->view.rowops = rd;
      }
    }
    double *dg_dev = nullptr;
    L->dinv = lalloc<T>(L, L->n, e, s);
    if (e == cudaSuccess) e = cudaMalloc(&dg_dev, L->n * sizeof(double));
    if (curved) {
      if (e == cudaSuccess) e = launch_curved_diagonal(v64, dg_dev, s);
    } else {
      std::vector<double> dg;
      laplace_diagonal(L->geo, M->basis64, dg);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dg_dev, dg.data(), dg.size() * sizeof(double), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e == cudaSuccess) { note_launch(); inv_kernel<T><<<mg_grid(L->n), 256, 0, s>>>(dg_dev, L->dinv, L->n); }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (dg_dev) cudaFree(dg_dev);
    const size_t nb = (size_t)L->n * H->cols;   // every column of the block of right-hand sides
    L->x = lalloc<T>(L, nb, e, s); L->b = lalloc<T>(L, nb, e, s); L->r = lalloc<T>(L, nb, e, s);
    L->d = lalloc<T>(L, nb, e, s); L->t = lalloc<T>(L, nb, e, s); L->z = lalloc<T>(L, L->n, e, s);
    L->x2 = lalloc<T>(L, nb, e, s);
    void *p = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&p, MS_COUNT * H->cols * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, MS_COUNT * H->cols * sizeof(double), s);
    if (e == cudaSuccess) { L->allocs.push_back(p); L->sc = (double *)p; }
    if (e == cudaSuccess) e = cudaMalloc(&p, MG_RED * H->cols * sizeof(double));
    if (e == cudaSuccess) { L->allocs.push_back(p); L->partial = (double *)p; }
    if (e == cudaSuccess) e = estimate_lmax(L, s);
    // next coarser level: the wall-normal direction alone while the thinnest cells are much
    // thinner than the in-plane spacing, otherwise every even direction. On such cells the
    // operator couples strongly along y and the Jacobi smoother reduces only errors that are
    // smooth along y, which full coarsening cannot represent (two-grid rate about 0.85 on the
    // graded channel; 0.55 with y-coarsening); semi-coarsening halves the CG iterations.
    int cf[3] = {nx % 2 == 0 ? 2 : 1, ny % 2 == 0 ? 2 : 1, nz % 2 == 0 ? 2 : 1};
    {
      double hymin = 1e300;
      for (int j = 0; j < ny; ++j) hymin = std::min(hymin, yv[j + 1] - yv[j]);
      const double hxz = std::min(M->P.lx / nx, M->P.lz / nz);
      if (ny % 2 == 0 && 2.0 * hymin <= kSemiRatio * hxz) cf[0] = cf[2] = 1;
    }
    const long cells = (long)nx * ny * nz;
    if (cells * 8 <= kDenseMax || cells <= 64 || (cf[0] == 1 && cf[1] == 1 && cf[2] == 1) || lev >= 12) break;
    XferDims X;
    X.fnx = nx; X.fny = ny; X.fnz = nz;
    X.cf[0] = cf[0]; X.cf[1] = cf[1]; X.cf[2] = cf[2];
    X.py = nullptr;
    if (cf[1] == 2) {
      // child rows 2J and 2J+1 of coarse row J split it in the ratio of their heights (boxes) or
      // at the middle of the logical coordinate (curved cells are images of the logical grid)
      const int cny = ny / 2, nn = n * n;
      std::vector<double> P((size_t)cny * 2 * nn);
      for (int J = 0; J < cny; ++J) {
        double r = 0.5;
        if (!curved) {
          const double h0 = yv[2 * J + 1] - yv[2 * J], h1 = yv[2 * J + 2] - yv[2 * J + 1];
          r = h0 / (h0 + h1);
        }
        embed_matrix(n, 0.0, r, &P[((size_t)J * 2 + 0) * nn]);
        embed_matrix(n, r, 1.0 - r, &P[((size_t)J * 2 + 1) * nn]);
      }
      std::vector<T> PT(P.begin(), P.end());
      T *pyd = lalloc<T>(L, PT.size(), e, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(pyd, PT.data(), PT.size() * sizeof(T), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      X.py = pyd;
    }
    nx /= cf[0]; ny /= cf[1]; nz /= cf[2];
    X.cnx = nx; X.cny = ny; X.cnz = nz;
    L->to_coarse = X;
    if (cf[1] == 2) {
      std::vector<double> yc(ny + 1);
      for (int j = 0; j <= ny; ++j) yc[j] = yv[2 * j];
      yv.swap(yc);
    }
  }
  if (e != cudaSuccess) return e;
  // coarsest level: dense solve at degree k, or one more level with Q_1 on the same cells solved
  // densely, or (too large for either) the iterative coarse PCG
  Lvl<T> *C = H->L.back();
  const long cells = (long)C->geo.nx * C->geo.ny * C->geo.nz;
  int kd = -1;
  if (C->n <= kDenseMax) kd = k;
  else if (k > 1 && cells * 8 <= kDenseMax) kd = 1;
  if (kd < 0) return e;
  Lvl<T> *D = C;
  Basis<double> b1d;
  const Basis<double> *Bd = &M->basis64;
  MeshView<double> d64 = v64;   // FP64 view of the dense level (curved)
  if (kd == 1) {
    D = new Lvl<T>();
    H->L.push_back(D);
    box_geometry(1, C->geo.nx, C->geo.ny, C->geo.nz, M->P.lx, M->P.lz, C->geo.yv, D->geo);
    D->n = cells * 8;
    fill_basis<double>(1, 2, M->P.q_wall, &b1d);
    Bd = &b1d;
    // transfer table P1 (n x 2): linear functions at the degree-k Gauss-Lobatto nodes
    std::vector<double> P1(2 * n);
    {
      double z[NMAX], w[NMAX];
      lobatto_nodes(n, z);
      (void)w;
      for (int i = 0; i < n; ++i) { P1[2 * i] = 1.0 - z[i]; P1[2 * i + 1] = z[i]; }
    }
    std::vector<T> P1T(P1.begin(), P1.end());
    T *p1d = lalloc<T>(C, P1T.size(), e, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p1d, P1T.data(), P1T.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    C->p1 = p1d;
    D->view = C->view;
    D->view.n1 = 2;
    D->view.np = D->n;
    D->x = lalloc<T>(D, (size_t)D->n * H->cols, e, s); D->b = lalloc<T>(D, (size_t)D->n * H->cols, e, s);
    void *p = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&p, MS_COUNT * H->cols * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, MS_COUNT * H->cols * sizeof(double), s);
    if (e == cudaSuccess) { D->allocs.push_back(p); D->sc = (double *)p; }
    if (e == cudaSuccess) e = cudaMalloc(&p, MG_RED * H->cols * sizeof(double));
    if (e == cudaSuccess) { D->allocs.push_back(p); D->partial = (double *)p; }
    if (curved) {
      // degree-1 tables and basis of the coarsest cells for the dense assembly
      CurvedHost cg;
      dgw_mesh_params Pl = M->P;
      Pl.full_quadrature = 0;
      curved_geometry(Pl, C->geo.nx, C->geo.ny, C->geo.nz, 1, b1d, cg);
      Lvl<double> tmp;
      d64.n1 = 2;
      d64.np = D->n;
      for (int t = 0; t < NQSET; ++t) d64.q[t] = b1d.q[t];
      double *bmem = lalloc<double>(&tmp, (sizeof(b1d) + sizeof(double) - 1) / sizeof(double), e, s);
      Basis<double> *bdev = reinterpret_cast<Basis<double> *>(bmem);
      if (e == cudaSuccess) e = cudaMemcpyAsync(bdev, &b1d, sizeof(b1d), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      d64.basis = bdev;
      upload_curved<double>(&tmp, cg, d64, e, s);
      D->allocs.insert(D->allocs.end(), tmp.allocs.begin(), tmp.allocs.end());
    }
  }
  if (e != cudaSuccess) return e;
  // assemble the level operator column by column, invert A + c 1 1^T
  const int N = (int)D->n;
  std::vector<double> A((size_t)N * N);
  if (curved) {
    e = assemble_device(d64, N, A, s);
    if (e != cudaSuccess) return e;
  } else {
    std::vector<double> rops;
    box_rowops(D->geo, *Bd, rops);
    std::vector<double> ej(N, 0.0), col(N);
    for (int jc = 0; jc < N; ++jc) {
      ej[jc] = 1.0;
      host_box_apply(D->geo, *Bd, rops, ej.data(), col.data());
      ej[jc] = 0.0;
      for (int i = 0; i < N; ++i) A[(size_t)i * N + jc] = col[i];
    }
  }
  T *ad = nullptr;
  if (!dense_inverse_device<T>(D, std::move(A), N, &ad, e, s)) return e;   // keep the iterative coarse solve
  D->ainv = ad;
  return e;
}

// Chebyshev smoothing with the point-Jacobi diagonal. Every step after a zero initial guess is one
// fused launch: the operator kernel applies A to the current iterate and, in its epilogue, updates
// the direction d and writes the next iterate into the other buffer (neighbouring cells still read
// the current one); the result ends in L->x.
template <typename T>
static void chebyshev(const Hierarchy<T> *H, Lvl<T> *L, bool zero_init, cudaStream_t s) {
  const double lmax = kLmaxSafety * L->lmax, lmin = lmax / kSmoothRange;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double rho = 1.0 / sigma;
  const int G = mg_grid(L->n), nc = H->ncols;
  T *cur = L->x;
  int k = 0;
  if (zero_init) {   // x = 0: the first step needs no operator apply
    note_launch();
    cheb_step<T><<<dim3(G, nc), 256, 0, s>>>(L->x, L->d, L->b, L->t, L->dinv, L->n, T(0), (T)(1.0 / theta), 1, 1);
    k = 1;
  }
  for (; k < H->cheb; ++k) {
    LapEpi<T> epi{};
    epi.mode = LAP_CHEB;
    epi.ncols = nc;
    epi.b = L->b;
    epi.d = L->d;
    epi.dinv = L->dinv;
    epi.xout = cur == L->x ? L->x2 : L->x;
    if (k == 0) {
      epi.c1 = T(0);
      epi.c2 = (T)(1.0 / theta);
      epi.first = 1;
    } else {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      epi.c1 = (T)(rho_new * rho);
      epi.c2 = (T)(2.0 * rho_new / delta);
      epi.first = 0;
      rho = rho_new;
    }
    launch_laplace_epi<T>(L->view, cur, nullptr, epi, s);
    cur = epi.xout;
  }
  if (cur != L->x) cudaMemcpyAsync(L->x, cur, (size_t)L->n * nc * sizeof(T), cudaMemcpyDeviceToDevice, s);
}

// Coarsest level: the dense (pseudo-)inverse for every column, or (one column only) the iterative
// coarse PCG.
template <typename T>
static void coarse_solve(const Hierarchy<T> *H, Lvl<T> *L, cudaStream_t s) {
  const long n = L->n;
  const int G = mg_grid(n), nc = H->ncols;
  if (L->ainv) {
    // consistent right-hand side, then the exact (pseudo-)inverse
    mg_reduce<T>(L->b, nullptr, n, L->partial, L->sc, MS_SUM, s, nc);
    note_launches(2);
    sub_mean_T<T><<<dim3(G, nc), 256, 0, s>>>(L->b, n, L->sc, MS_SUM);
    dense_gemv<T><<<dim3((int)((n * 32 + 255) / 256), nc), 256, 0, s>>>(L->ainv, L->b, L->x, (int)n);
    return;
  }
  cudaMemsetAsync(L->x, 0, n * sizeof(T), s);
  // the coarse problem is singular (constants): make its right-hand side consistent
  mg_reduce<T>(L->b, nullptr, n, L->partial, L->sc, MS_SUM, s);
  note_launch();
  sub_mean_T<T><<<G, 256, 0, s>>>(L->b, n, L->sc, MS_SUM);
  cudaMemcpyAsync(L->r, L->b, n * sizeof(T), cudaMemcpyDeviceToDevice, s);
  for (int it = 0; it < kCoarseIters; ++it) {
    note_launch();
    cpcg_precond<T><<<G, 256, 0, s>>>(L->z, L->r, L->dinv, n);
    mg_reduce<T>(L->z, nullptr, n, L->partial, L->sc, MS_SUM, s);
    note_launch();
    sub_mean_T<T><<<G, 256, 0, s>>>(L->z, n, L->sc, MS_SUM);
    mg_reduce<T>(L->r, L->z, n, L->partial, L->sc, MS_RZNEW, s);
    note_launch();
    cpcg_direction<T><<<G, 256, 0, s>>>(L->d, L->z, n, L->sc, it == 0);
    note_launch();
    shift_scalar<<<1, 32, 0, s>>>(L->sc, MS_RZ, MS_RZNEW);
    launch_laplace<T>(L->view, L->d, L->t, s);
    mg_reduce<T>(L->d, L->t, n, L->partial, L->sc, MS_DQ, s);
    note_launch();
    cpcg_update<T><<<G, 256, 0, s>>>(L->x, L->r, L->d, L->t, n, L->sc);
  }
}

template <typename T>
static void vcycle(const Hierarchy<T> *H, size_t lev, cudaStream_t s) {
  Lvl<T> *L = H->L[lev];
  const int nc = H->ncols;
  if (lev + 1 == H->L.size()) {
    coarse_solve(H, L, s);
    return;
  }
  Lvl<T> *C = H->L[lev + 1];
  chebyshev(H, L, true, s);
  LapEpi<T> res{};
  res.mode = LAP_RESIDUAL;
  res.b = L->b;
  res.ncols = nc;
  launch_laplace_epi<T>(L->view, L->x, L->r, res, s);   // r = b - A x
  note_launch();
  if (L->p1) p_restrict<T><<<dim3(L->view.nc, nc), 64, 0, s>>>(L->p1, L->view.n1, L->r, C->b);
  else launch_restrict<T>(H->basis, L->to_coarse, L->view.n1, L->r, C->b, C->view.nc, s, nc);
  vcycle(H, lev + 1, s);
  note_launch();
  if (L->p1) p_prolongate_add<T><<<dim3(L->view.nc, nc), 64, 0, s>>>(L->p1, L->view.n1, C->x, L->x);
  else launch_prolong<T>(H->basis, L->to_coarse, L->view.n1, C->x, L->x, C->view.nc, s, nc);
  chebyshev(H, L, false, s);
}

cudaError_t mg_setup(dgw_mesh *M, dgw_solver *S, int mode, int cheb, cudaStream_t s) {
  if (S->mg_ready && S->mg_mode == mode && S->mg_cheb == cheb) return cudaSuccess;
  mg_free(S);
  if (S->vgraph) { cudaGraphExecDestroy(S->vgraph); S->vgraph = nullptr; }
  if (S->vgraph32) { cudaGraphExecDestroy(S->vgraph32); S->vgraph32 = nullptr; }
  MGLevel *ml = new MGLevel();
  cudaError_t e;
  if (mode == 1) {
    auto *H = new Hierarchy<float>();
    H->cheb = cheb;
    H->basis = M->v32.basis;
    ml->prec = 1;
    ml->h = H;
    e = build_hierarchy<float>(M, H, M->v32, nullptr, s);
  } else {
    auto *H = new Hierarchy<double>();
    H->cheb = cheb;
    H->basis = M->v64.basis;
    ml->prec = 0;
    ml->h = H;
    e = build_hierarchy<double>(M, H, M->v64, nullptr, s);
  }
  S->levels.push_back(ml);
  if (e != cudaSuccess) { mg_free(S); return e; }
  S->mg_ready = true;
  S->mg_mode = mode;
  S->mg_cheb = cheb;
  return cudaSuccess;
}

cudaError_t mg_vcycle(dgw_mesh *M, dgw_solver *S, int mode, const double *r, double *z, cudaStream_t s) {
  (void)mode;
  MGLevel *ml = S->levels.empty() ? nullptr : S->levels[0];
  if (!ml) return cudaErrorNotReady;
  const long n = M->np;
  const int G = mg_grid(n);
  if (ml->prec == 1) {
    auto *H = (Hierarchy<float> *)ml->h;
    note_launch();
    scale_in<float><<<G, 256, 0, s>>>(H->L[0]->b, r, n, S->sc, SC_RR);
    vcycle(H, 0, s);
    note_launch();
    scale_out<float><<<G, 256, 0, s>>>(z, H->L[0]->x, n, S->sc, SC_RR);
  } else {
    auto *H = (Hierarchy<double> *)ml->h;
    note_launch();
    scale_in<double><<<G, 256, 0, s>>>(H->L[0]->b, r, n, S->sc, SC_RR);
    vcycle(H, 0, s);
    note_launch();
    scale_out<double><<<G, 256, 0, s>>>(z, H->L[0]->x, n, S->sc, SC_RR);
  }
  return cudaGetLastError();
}

cudaError_t mg_level0_f32(dgw_solver *S, float **b0, float **x0) {
  MGLevel *ml = S->levels.empty() ? nullptr : S->levels[0];
  if (!ml || ml->prec != 1) return cudaErrorNotReady;
  auto *H = (Hierarchy<float> *)ml->h;
  *b0 = H->L[0]->b;
  *x0 = H->L[0]->x;
  return cudaSuccess;
}

cudaError_t mg_vcycle_f32(dgw_solver *S, cudaStream_t s) {
  MGLevel *ml = S->levels.empty() ? nullptr : S->levels[0];
  if (!ml || ml->prec != 1) return cudaErrorNotReady;
  vcycle((Hierarchy<float> *)ml->h, 0, s);
  return cudaGetLastError();
}

// FP32 hierarchy over a block of cols right-hand sides (box cells, dense coarsest solve): the
// batched mixed-precision solve runs one V-cycle for every column at once.
cudaError_t mg_batch_create(dgw_mesh *M, int cols, int cheb, cudaStream_t s, void **out) {
  *out = nullptr;
  if (M->P.geometry != 0 || !M->has32 || cols < 1) return cudaErrorNotSupported;
  auto *H = new Hierarchy<float>();
  H->cheb = cheb;
  H->basis = M->v32.basis;
  H->cols = cols;
  H->ncols = 1;
  cudaError_t e = build_hierarchy<float>(M, H, M->v32, nullptr, s);
  if (e == cudaSuccess && !H->L.back()->ainv) e = cudaErrorNotSupported;   // the iterative coarse solve is one column
  if (e != cudaSuccess) {
    free_hier(H);
    return e;
  }
  *out = H;
  return cudaSuccess;
}

void mg_batch_free(void *h) { free_hier(static_cast<Hierarchy<float> *>(h)); }

void mg_batch_level0(void *h, float **b0, float **x0) {
  auto *H = static_cast<Hierarchy<float> *>(h);
  *b0 = H->L[0]->b;
  *x0 = H->L[0]->x;
}

cudaError_t mg_batch_vcycle(void *h, int ncols, cudaStream_t s) {
  auto *H = static_cast<Hierarchy<float> *>(h);
  if (ncols < 1 || ncols > H->cols) return cudaErrorInvalidValue;
  H->ncols = ncols;
  vcycle(H, 0, s);
  H->ncols = 1;
  return cudaGetLastError();
}

int mg_describe(dgw_solver *S, double *lmax, int *cells, int max_levels) {
  if (S->levels.empty()) return 0;
  MGLevel *ml = S->levels[0];
  int nl = 0;
  auto fill = [&](auto *H) {
    for (auto *L : H->L) {
      if (nl < max_levels) {
        if (lmax) lmax[nl] = L->lmax;
        if (cells) cells[nl] = L->view.nc;
      }
      ++nl;
    }
  };
  if (ml->prec == 1) fill((Hierarchy<float> *)ml->h);
  else fill((Hierarchy<double> *)ml->h);
  return nl;
}

int mg_levels(dgw_solver *S) {
  if (S->levels.empty()) return 0;
  MGLevel *ml = S->levels[0];
  return ml->prec == 1 ? (int)((Hierarchy<float> *)ml->h)->L.size() : (int)((Hierarchy<double> *)ml->h)->L.size();
}

void mg_free(dgw_solver *S) {
  for (MGLevel *ml : S->levels) {
    if (ml->prec == 1) free_hier((Hierarchy<float> *)ml->h);
    else if (ml->prec == 0) free_hier((Hierarchy<double> *)ml->h);
    delete ml;
  }
  S->levels.clear();
  S->mg_ready = false;
  S->mg_mode = -1;
}

}  // namespace dgw
