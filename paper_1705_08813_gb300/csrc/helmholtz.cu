// Velocity mass operator and the viscous Helmholtz solve of the dual-splitting step
// (Sec. 4.2 mass term; eq. helmholtzspat): (gamma M + V) u = rhs with gamma = gamma_0 / dt and
// V u = -F^nu(vbar, v~; ubar, u~) with the frozen nu_t of the last eddy-viscosity update. The
// operator is not symmetric (the adjoint-consistency terms of eq. viscous_multiscale), so the solve
// is restarted GMRES with right preconditioning (Sec. 5: "the GMRES solver of the Helmholtz
// equation"), in FP64.
//
// Preconditioner: the block-diagonal inverse of gamma M per cell. With the k+1 Gauss points the
// standard part of a cell's mass matrix is S^T W S per component (S = S_1 (x) S_1 (x) S_1 the square
// node-to-point interpolation, W the diagonal of |det J| w at the points), so its inverse is
// S^-1 W^-1 S^-T: six 1-D passes of S_1^-1 and a pointwise division, exact on boxes and on curved
// cells off the wall (wall cells integrate with q_w points across the wall; there it is exact only
// where det J is constant). The enriched DoFs of a wall cell (8 per component with l = 1, one with
// l = 0) take the inverse of their own block, computed once from the mass operator. The coupling
// between standard and enriched DoFs is left to GMRES: an exact block inverse through the Schur
// complement Mee - Mes Mss^-1 Mse gained nothing on the flat channel and, where Mss^-1 is only
// approximate (wall cells of curved geometry, q_w points across the wall and a non-constant det J),
// turned the nearly singular complement indefinite and stalled GMRES.
//
// Orthogonalisation: classical Gram-Schmidt applied twice, so each Krylov step needs two batched
// reductions (all inner products at once) and one norm, deterministic two-stage sums.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dgw_internal.h"

struct dgw_helm {
  int m = 0;                       // restart length the basis was allocated for
  double *V = nullptr, *Z = nullptr;   // (m+1) and m vectors of n_u
  double *w = nullptr, *t = nullptr, *r = nullptr;
  double *partial = nullptr, *h = nullptr, *host_h = nullptr;
  double *vol = nullptr;           // [nc] cell volumes
  double *detw = nullptr;          // [nc][(k+1)^3] |det J| w at the Gauss points
  double *meeinv = nullptr;        // [ne][8][8] inverse enriched mass blocks
  double *m1inv = nullptr;         // [n][n] S_1^-1, inverse of the 1-D node-to-Gauss-point interpolation
  double minv1[dgw::NMAX * dgw::NMAX] = {};  // host copy of the inverse 1-D mass matrix (S_1^T W S_1)^-1
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace dgw {

namespace {

constexpr int kBlocks = 304;     // 2 x 152 SMs
constexpr int kThreads = 256;
constexpr int kMaxRestart = 64;

__device__ double block_sum_d(double v) {
  __shared__ double part[32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) part[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  }
  __syncthreads();
  return s;
}

// partial[i][block] = sum_k V_i[k] w[k] for i < nv (blockIdx.y = i)
__global__ void multidot_partial(const double *__restrict__ V, const double *__restrict__ w, long n, int nv,
                                 double *__restrict__ partial) {
  const int i = blockIdx.y;
  const double *v = V + (size_t)i * n;
  double s = 0.0;
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) s += v[k] * w[k];
  s = block_sum_d(s);
  if (threadIdx.x == 0) partial[(size_t)i * gridDim.x + blockIdx.x] = s;
}

// h[i] = sum of partial[i][*] (one warp per i, fixed order)
__global__ void multidot_finish(const double *__restrict__ partial, int nb, int nv, double *__restrict__ h) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) s += partial[(size_t)i * nb + b];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (threadIdx.x == 0) h[i] = s;
}

// w -= sum_{i < nv} h[i] V_i
__global__ void subtract_projections(double *__restrict__ w, const double *__restrict__ V, const double *__restrict__ h,
                                     long n, int nv) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    double s = w[k];
    for (int i = 0; i < nv; ++i) s -= h[i] * V[(size_t)i * n + k];
    w[k] = s;
  }
}

__global__ void scale_into(double *__restrict__ y, const double *__restrict__ x, double a, long n) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) y[k] = a * x[k];
}

// y = a x + y
__global__ void axpy_kernel(double *__restrict__ y, const double *__restrict__ x, double a, long n) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) y[k] += a * x[k];
}

// y = rhs - (gamma t + y) with t = M x, y = V x on input
__global__ void residual_kernel(double *__restrict__ y, const double *__restrict__ rhs, const double *__restrict__ t,
                                double gamma, long n) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
    y[k] = rhs[k] - (gamma * t[k] + y[k]);
}

// y = gamma t + y (the Helmholtz operator from the mass and viscous applies)
__global__ void combine_kernel(double *__restrict__ y, const double *__restrict__ t, double gamma, long n) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
    y[k] += gamma * t[k];
}

// out = s Mss^-1 in for one cell and component: S^-1 W^-1 S^-T by six 1-D passes of Si = S_1^-1 and a
// pointwise division by w = |det J| w (A, Bs: shared scratch of n^3). Ends with a barrier.
__device__ void mss_inverse(const double *in, double *out, const double *Si, const double *w, double s, int n,
                            double *A, double *Bs) {
  const int nn = n * n, n3 = nn * n;
  auto pass = [&](const double *src, double *dst, int ax, bool tr) {
    const int st = ax == 0 ? 1 : (ax == 1 ? n : nn);
    for (int t = threadIdx.x; t < n3; t += blockDim.x) {
      const int i = (t / st) % n, base = t - i * st;
      double v = 0.0;
      for (int b = 0; b < n; ++b) v += (tr ? Si[b * n + i] : Si[i * n + b]) * src[base + b * st];
      dst[t] = v;
    }
    __syncthreads();
  };
  for (int t = threadIdx.x; t < n3; t += blockDim.x) A[t] = in[t];
  __syncthreads();
  pass(A, Bs, 0, true);
  pass(Bs, A, 1, true);
  pass(A, Bs, 2, true);
  for (int t = threadIdx.x; t < n3; t += blockDim.x) Bs[t] *= s / w[t];
  __syncthreads();
  pass(Bs, A, 0, false);
  pass(A, Bs, 1, false);
  pass(Bs, A, 2, false);
  for (int t = threadIdx.x; t < n3; t += blockDim.x) out[t] = A[t];
  __syncthreads();
}

// z = (gamma M_blocks)^-1 r, one CTA per cell: Mss^-1 per component, and the nef x nef enriched
// block inverse of each component in wall cells.
// One CTA per cell of rows [0, rb) and [rt, ny) (rb = rt = ny: every row), x fastest.
__global__ void inverse_mass_kernel(const double *__restrict__ r, double *__restrict__ z, const double *__restrict__ sinv,
                                    const double *__restrict__ detw, const int *__restrict__ enr,
                                    const int *__restrict__ slot, const double *__restrict__ meeinv, int n, int nef,
                                    long np, double inv_gamma, int nx, int ny, int rb, int rt) {
  __shared__ double A[NMAX * NMAX * NMAX], Bs[NMAX * NMAX * NMAX], Si[NMAX * NMAX];
  int c;
  {
    const int nr = rb + (ny - rt), b = blockIdx.x;
    const int i = b % nx, rr = (b / nx) % nr, kz = b / (nx * nr);
    c = i + nx * ((rr < rb ? rr : rt + (rr - rb)) + ny * kz);
  }
  const int n3 = n * n * n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) Si[t] = sinv[t];
  __syncthreads();
  for (int a = 0; a < 3; ++a)
    mss_inverse(r + ((size_t)c * 3 + a) * n3, z + ((size_t)c * 3 + a) * n3, Si, detw + (size_t)c * n3, inv_gamma, n,
                A, Bs);
  const int e = enr ? enr[c] : -1;
  if (e < 0 && slot && slot[c] >= 0) {   // wall model switched off here: zero coefficients
    for (int t = threadIdx.x; t < 3 * nef; t += blockDim.x) z[3 * np + (size_t)slot[c] * 3 * nef + t] = 0.0;
    return;
  }
  if (e < 0 || threadIdx.x >= 3 * nef) return;
  const int a = threadIdx.x / nef, v = threadIdx.x % nef;
  const double *rin = r + 3 * np + ((size_t)e * 3 + a) * nef;
  double acc = 0.0;
  for (int w = 0; w < nef; ++w) acc += meeinv[(size_t)e * 64 + v * nef + w] * rin[w];
  z[3 * np + ((size_t)e * 3 + a) * nef + v] = inv_gamma * acc;
}

// The inverse 1-D mass matrix as a kernel parameter (read from the constant parameter bank).
struct Minv1 {
  double m[NMAX * NMAX];
};

// z = scale M_c^-1 r on standard box cells: the cell mass matrix is V (M_1 x M_1 x M_1), so its inverse is
// (M_1^-1 x M_1^-1 x M_1^-1) / V, three line passes instead of the six of S^-1 W^-1 S^-T. cpb cells of
// one row per CTA (rows [j0, j0 + nrows)), one line of one cell per thread, passes in place.
template <int K>
__global__ void __launch_bounds__(128) inverse_mass_box_kernel(const double *__restrict__ r, double *__restrict__ z, Minv1 Mi,
                                                               int nx, int ny, const double *__restrict__ hy, double hx,
                                                               double hz, int cpb, int j0, int nrows, double scale) {
  constexpr int n = K + 1, n2 = n * n, n3 = n2 * n;
  extern __shared__ __align__(16) double X[];   // cpb x 3 x n3
  const int segs = nx / cpb, b = blockIdx.x;
  const int i0 = (b % segs) * cpb, j = j0 + (b / segs) % nrows, kz = b / (segs * nrows);
  const size_t o = ((size_t)i0 + (size_t)nx * (j + (size_t)ny * kz)) * 3 * n3;
  for (int t = threadIdx.x; t < cpb * 3 * n3; t += blockDim.x) X[t] = r[o + t];
  __syncthreads();
  const double sv = scale / (hx * hy[j] * hz);
  const int tid = threadIdx.x;
  const bool line = tid < cpb * n2;
  const int cl = line ? tid / n2 : 0, l = line ? tid - cl * n2 : 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (line) {
      const int base = d == 0 ? n * l : (d == 1 ? (l % n) + n2 * (l / n) : l);
      const int st = d == 0 ? 1 : (d == 1 ? n : n2);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double *xl = X + (cl * 3 + a) * n3 + base;
        double v[n];
#pragma unroll
        for (int q = 0; q < n; ++q) v[q] = xl[q * st];
#pragma unroll
        for (int q = 0; q < n; ++q) {
          double acc = 0.0;
#pragma unroll
          for (int p = 0; p < n; ++p) acc = fma(Mi.m[q * n + p], v[p], acc);
          xl[q * st] = d == 2 ? sv * acc : acc;
        }
      }
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < cpb * 3 * n3; t += blockDim.x) z[o + t] = X[t];
}

template <int K>
cudaError_t launch_imass_box_k(dgw_mesh *M, const Minv1 &Mi, const double *r, double *z, double scale, cudaStream_t s) {
  const MeshView<double> &m = M->v64;
  constexpr int n = K + 1, n2 = n * n, n3 = n2 * n;
  int cpb = 1;
  while (cpb * 2 <= 8 && cpb * 2 * n2 <= 128 && m.nx % (cpb * 2) == 0) cpb *= 2;
  const int nrows = m.std_hi - m.std_lo, threads = ((cpb * n2 + 31) / 32) * 32;
  note_launch();
  inverse_mass_box_kernel<K><<<(m.nx / cpb) * nrows * m.nz, threads, (size_t)cpb * 3 * n3 * sizeof(double), s>>>(
      r, z, Mi, m.nx, m.ny, m.hy, m.hx, m.hz, cpb, m.std_lo, nrows, scale);
  return cudaGetLastError();
}

// z = scale M^-1 r in every cell without switched-on enrichment (exact there) and the block-diagonal
// approximation in cells with the wall model on: the box kernel on the channel rows without
// enrichment slots, the general kernel on the other rows (all of them on curved meshes)
cudaError_t launch_inverse_mass(dgw_mesh *M, const double *r, double *z, double scale, cudaStream_t s) {
  const dgw_helm *H = M->helm;
  const MeshView<double> &m = M->v64;
  int rb = m.ny, rt = m.ny;
  if (m.geo == GEO_BOX && m.std_hi > m.std_lo) {
    Minv1 Mi;
    std::memcpy(Mi.m, H->minv1, sizeof(Mi.m));
    cudaError_t e = cudaErrorInvalidValue;
    switch (M->n1) {
      case 2: e = launch_imass_box_k<1>(M, Mi, r, z, scale, s); break;
      case 3: e = launch_imass_box_k<2>(M, Mi, r, z, scale, s); break;
      case 4: e = launch_imass_box_k<3>(M, Mi, r, z, scale, s); break;
      case 5: e = launch_imass_box_k<4>(M, Mi, r, z, scale, s); break;
      case 6: e = launch_imass_box_k<5>(M, Mi, r, z, scale, s); break;
    }
    if (e != cudaSuccess) return e;
    rb = m.std_lo;
    rt = m.std_hi;
  }
  const int nr = rb + (m.ny - rt);
  if (nr <= 0) return cudaSuccess;
  note_launch();
  inverse_mass_kernel<<<m.nx * nr * m.nz, 128, 0, s>>>(r, z, H->m1inv, H->detw, m.enr, m.slot, H->meeinv, M->n1, M->nef,
                                                       M->np, scale, m.nx, m.ny, rb, rt);
  return cudaGetLastError();
}

// detw[c][q] = |det J| w_q at the Gauss points: boxes vol_c w0 w1 w2, curved cells from the metric
// records (the map is an extrusion along z, so det J depends on (q0, q1) and the cell's column)
__global__ void detw_kernel(MeshView<double> m, const double *__restrict__ vol, double *__restrict__ detw) {
  const Basis<double> &B = *m.basis;
  const int n = m.n1, n3 = n * n * n, q = B.q[QSET_LIN];
  const long total = (long)m.nc * n3;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
    const int c = (int)(g / n3), t = (int)(g % n3);
    const int i0 = t % n, i1 = (t / n) % n, i2 = t / (n * n);
    const double w3 = B.w[QSET_LIN][i0] * B.w[QSET_LIN][i1] * B.w[QSET_LIN][i2];
    double d = vol[c];
    if (m.geo == GEO_CURVED) d = fabs(m.mvol[0][((size_t)(c % (m.nx * m.ny)) * q * q + i0 + q * i1) * MREC + 9]);
    detw[g] = d * w3;
  }
}

// vol[c] = sum of the cell's component-0 standard outputs of M applied to u = e_x (partition of unity)
__global__ void cell_sum_kernel(const double *__restrict__ y, int n3, double *__restrict__ vol) {
  const int c = blockIdx.x;
  double s = 0.0;
  for (int t = threadIdx.x; t < n3; t += blockDim.x) s += y[(size_t)c * 3 * n3 + t];
  s = block_sum_d(s);
  if (threadIdx.x == 0) vol[c] = s;
}

// u[3 np + (e*3 + 0)*nef + v] = 1 for every enriched cell e (component x, weight v)
__global__ void enriched_unit_kernel(double *__restrict__ u, long np, int ne, int nef, int v) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x)
    u[3 * np + (size_t)e * 3 * nef + v] = 1.0;
}

inline int grid_for(long n) {
  long g = (n + 255) / 256;
  return (int)std::min<long>(std::max<long>(g, 1), 152 * 16);
}

// inverse of an SPD q x q matrix (q <= 8, row-major) by Gauss-Jordan elimination without pivoting
// (host); false if a pivot is not positive
bool invert_spd(const double *A, double *inv, int q) {
  double a[8][16];
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < 2 * q; ++j) a[i][j] = j < q ? A[i * q + j] : (j - q == i ? 1.0 : 0.0);
  for (int k = 0; k < q; ++k) {
    const double p = a[k][k];
    if (!(p > 0.0)) return false;
    for (int j = 0; j < 2 * q; ++j) a[k][j] /= p;
    for (int i = 0; i < q; ++i)
      if (i != k) {
        const double f = a[i][k];
        for (int j = 0; j < 2 * q; ++j) a[i][j] -= f * a[k][j];
      }
  }
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) inv[i * q + j] = a[i][q + j];
  return true;
}

}  // namespace

static void helm_free(dgw_helm *H) {
  if (!H) return;
  cudaFree(H->V); cudaFree(H->Z); cudaFree(H->w); cudaFree(H->t); cudaFree(H->r);
  cudaFree(H->partial); cudaFree(H->h); cudaFree(H->vol); cudaFree(H->detw); cudaFree(H->meeinv);
  cudaFree(H->m1inv);
  if (H->host_h) cudaFreeHost(H->host_h);
  if (H->ev_in) cudaEventDestroy(H->ev_in);
  if (H->ev_out) cudaEventDestroy(H->ev_out);
  if (H->stream) cudaStreamDestroy(H->stream);
  delete H;
}

// Workspace, cell volumes, 1-D inverse mass and the enriched inverse blocks (first use, and
// again when a larger restart length is asked for).
static cudaError_t helm_setup(dgw_mesh *M, int restart) {
  dgw_helm *H = M->helm;
  if (H && H->m >= restart) return cudaSuccess;
  if (H) { helm_free(H); M->helm = nullptr; }
  H = new dgw_helm();
  M->helm = H;
  const long nu = M->nu;
  const int n = M->n1;
  cudaError_t e = cudaStreamCreateWithFlags(&H->stream, cudaStreamNonBlocking);
  cudaStream_t s = H->stream;
  auto alloc = [&](double **p, size_t count) {
    if (e == cudaSuccess) e = cudaMalloc(p, std::max<size_t>(count, 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, std::max<size_t>(count, 1) * sizeof(double), s);
  };
  alloc(&H->V, (size_t)(restart + 1) * nu);
  alloc(&H->Z, (size_t)restart * nu);
  alloc(&H->w, nu);
  alloc(&H->t, nu);
  alloc(&H->r, nu);
  alloc(&H->partial, (size_t)(kMaxRestart + 1) * kBlocks);
  alloc(&H->h, kMaxRestart + 1);
  alloc(&H->vol, M->nc);
  alloc(&H->detw, (size_t)M->nc * n * n * n);
  alloc(&H->meeinv, (size_t)std::max(M->ne, 1) * 64);
  alloc(&H->m1inv, (size_t)n * n);
  if (e == cudaSuccess) e = cudaMallocHost(&H->host_h, (kMaxRestart + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&H->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&H->ev_out, cudaEventDisableTiming);
  if (e != cudaSuccess) return e;
  H->m = restart;
  // S_1^-1: inverse of the 1-D interpolation S_1[q][j] = l_j(x_q) (square, k+1 Gauss points and
  // Gauss-Lobatto nodes), Gauss-Jordan with partial pivoting on the host
  {
    std::vector<double> a((size_t)n * 2 * n, 0.0);
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) a[(size_t)i * 2 * n + j] = M->basis64.S[QSET_LIN][i * n + j];
      a[(size_t)i * 2 * n + n + i] = 1.0;
    }
    for (int k = 0; k < n; ++k) {
      int pr = k;
      for (int i = k + 1; i < n; ++i)
        if (std::fabs(a[(size_t)i * 2 * n + k]) > std::fabs(a[(size_t)pr * 2 * n + k])) pr = i;
      if (pr != k)
        for (int j = 0; j < 2 * n; ++j) std::swap(a[(size_t)k * 2 * n + j], a[(size_t)pr * 2 * n + j]);
      const double p = a[(size_t)k * 2 * n + k];
      for (int j = 0; j < 2 * n; ++j) a[(size_t)k * 2 * n + j] /= p;
      for (int i = 0; i < n; ++i)
        if (i != k) {
          const double f = a[(size_t)i * 2 * n + k];
          for (int j = 0; j < 2 * n; ++j) a[(size_t)i * 2 * n + j] -= f * a[(size_t)k * 2 * n + j];
        }
    }
    std::vector<double> inv((size_t)n * n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) inv[(size_t)i * n + j] = a[(size_t)i * 2 * n + n + j];
    e = cudaMemcpyAsync(H->m1inv, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    // (S_1^T W S_1)^-1 = S_1^-1 W^-1 S_1^-T for the box cells' inverse mass
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int q = 0; q < n; ++q) acc += inv[(size_t)i * n + q] * inv[(size_t)j * n + q] / M->basis64.w[QSET_LIN][q];
        H->minv1[i * n + j] = acc;
      }
  }
  // cell volumes: M e_x summed over each cell's component-x outputs
  const long np = M->np;
  if (e == cudaSuccess) {
    // component x of every cell = 1 (the first n3 of each cell's 3 n3 block); H->w starts zeroed
    std::vector<double> ex((size_t)3 * np, 0.0);
    const int n3 = n * n * n;
    for (long c = 0; c < M->nc; ++c)
      for (int i = 0; i < n3; ++i) ex[(size_t)c * 3 * n3 + i] = 1.0;
    e = cudaMemcpyAsync(H->w, ex.data(), ex.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = launch_vector_op<double>(OP_MASS, M->v64, H->w, H->t, s);
    if (e == cudaSuccess) {
      note_launches(2);
      cell_sum_kernel<<<M->nc, 128, 0, s>>>(H->t, n3, H->vol);
      detw_kernel<<<1216, 256, 0, s>>>(M->v64, H->vol, H->detw);
      e = cudaGetLastError();
    }
    // the tables are read on other streams too (the exact inverse mass): finish them here
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  // enriched blocks: M applied to the enrichment unit vectors of component x; the nef x nef blocks
  // are inverted on the host (stored with a stride of 64 per wall cell)
  if (e == cudaSuccess && M->ne > 0) {
    const int q = M->nef;
    std::vector<double> mee((size_t)M->ne * 64), inv((size_t)M->ne * 64), out(3 * (size_t)q * M->ne);
    for (int v = 0; v < q && e == cudaSuccess; ++v) {
      e = cudaMemsetAsync(H->w, 0, nu * sizeof(double), s);
      if (e == cudaSuccess) {
        note_launch();
        enriched_unit_kernel<<<(M->ne + 255) / 256, 256, 0, s>>>(H->w, np, M->ne, q, v);
        e = launch_vector_op<double>(OP_MASS, M->v64, H->w, H->t, s);
      }
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(out.data(), H->t + 3 * np, out.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      for (int c = 0; c < M->ne && e == cudaSuccess; ++c)
        for (int wv = 0; wv < q; ++wv) mee[(size_t)c * 64 + wv * q + v] = out[(size_t)c * 3 * q + wv];
    }
    for (int c = 0; c < M->ne && e == cudaSuccess; ++c) {
      bool zero = true;   // a switched-off cell has no enrichment functions: its block is zero
      for (int i = 0; i < q * q; ++i) zero = zero && mee[(size_t)c * 64 + i] == 0.0;
      if (zero) continue;
      if (!invert_spd(&mee[(size_t)c * 64], &inv[(size_t)c * 64], q)) e = cudaErrorInvalidValue;
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(H->meeinv, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  return e;
}

// t = M x, y = gamma t + V x
static cudaError_t helm_apply(dgw_mesh *M, double gamma, const double *x, double *y, double *t, cudaStream_t s) {
  cudaError_t e = launch_vector_op<double>(OP_MASS, M->v64, x, t, s);
  if (e == cudaSuccess) e = launch_vector_op<double>(OP_VISC, M->v64, x, y, s);
  if (e == cudaSuccess) {
    note_launch();
    combine_kernel<<<grid_for(M->nu), 256, 0, s>>>(y, t, gamma, M->nu);
    e = cudaGetLastError();
  }
  return e;
}

// h[0..nv) = V_i . w (on the host after the call)
static cudaError_t multidot(dgw_helm *H, const double *V, const double *w, long n, int nv, double *host,
                            cudaStream_t s) {
  note_launches(2);
  multidot_partial<<<dim3(kBlocks, nv), kThreads, 0, s>>>(V, w, n, nv, H->partial);
  multidot_finish<<<nv, 32, 0, s>>>(H->partial, kBlocks, nv, H->h);
  cudaError_t e = cudaMemcpyAsync(host, H->h, nv * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

dgw_status helmholtz_solve(dgw_mesh *M, double gamma, const double *rhs, double *u, const dgw_helmholtz_opts *o,
                           dgw_solve_info *info, cudaStream_t cs) {
  const int m = o->restart > 0 ? std::min(o->restart, kMaxRestart) : 30;
  cudaError_t e = helm_setup(M, m);
  if (e != cudaSuccess) return cuda_check(e, "dgw_helmholtz_solve: setup");
  dgw_helm *H = M->helm;
  cudaStream_t s = H->stream;
  cudaEventRecord(H->ev_in, cs);
  cudaStreamWaitEvent(s, H->ev_in, 0);
  const long nu = M->nu;
  const int G = grid_for(nu);
  const auto t0 = std::chrono::steady_clock::now();
  const unsigned long long dof0 = dof_counter();
  double *hh = H->host_h;
  // ||rhs||
  e = multidot(H, rhs, rhs, nu, 1, hh, s);
  if (e != cudaSuccess) return cuda_check(e, "dgw_helmholtz_solve");
  const double bnorm = std::sqrt(hh[0]);
  if (bnorm == 0.0) {
    cudaMemsetAsync(u, 0, nu * sizeof(double), s);
    cudaStreamSynchronize(s);
    info->iterations = 0;
    info->rel_residual = 0.0;
    info->ms = 0.0f;
    info->dof_applies = 0.0;
    return DGW_OK;
  }
  std::vector<double> Hm((size_t)(m + 1) * m, 0.0), cs_(m), sn(m), g(m + 1), y(m);
  int it = 0;
  double rel = 1.0;
  dgw_status st = DGW_OK;
  for (;;) {
    // r = rhs - (gamma M u + V u)
    e = launch_vector_op<double>(OP_MASS, M->v64, u, H->t, s);
    if (e == cudaSuccess) e = launch_vector_op<double>(OP_VISC, M->v64, u, H->r, s);
    if (e != cudaSuccess) return cuda_check(e, "dgw_helmholtz_solve: operator");
    note_launch();
    residual_kernel<<<G, 256, 0, s>>>(H->r, rhs, H->t, gamma, nu);
    e = multidot(H, H->r, H->r, nu, 1, hh, s);
    if (e != cudaSuccess) return cuda_check(e, "dgw_helmholtz_solve");
    const double beta = std::sqrt(std::max(hh[0], 0.0));
    rel = beta / bnorm;
    if (rel <= o->rtol) break;
    if (it >= o->max_iter) { st = DGW_ENOTCONV; break; }
    note_launch();
    scale_into<<<G, 256, 0, s>>>(H->V, H->r, 1.0 / beta, nu);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    for (; j < m && it < o->max_iter; ++j) {
      double *Vj = H->V + (size_t)j * nu, *Zj = H->Z + (size_t)j * nu, *Vn = H->V + (size_t)(j + 1) * nu;
      e = launch_inverse_mass(M, Vj, Zj, 1.0 / gamma, s);
      if (e == cudaSuccess) e = helm_apply(M, gamma, Zj, H->w, H->t, s);
      if (e != cudaSuccess) return cuda_check(e, "dgw_helmholtz_solve: operator");
      // classical Gram-Schmidt, twice
      std::vector<double> hcol(j + 2, 0.0);
      for (int pass = 0; pass < 2; ++pass) {
        e = multidot(H, H->V, H->w, nu, j + 1, hh, s);
        if (e != cudaSuccess) return cuda_check(e, "dgw_helmholtz_solve");
        for (int i = 0; i <= j; ++i) hcol[i] += hh[i];
        note_launch();
        subtract_projections<<<G, 256, 0, s>>>(H->w, H->V, H->h, nu, j + 1);
      }
      e = multidot(H, H->w, H->w, nu, 1, hh, s);
      if (e != cudaSuccess) return cuda_check(e, "dgw_helmholtz_solve");
      hcol[j + 1] = std::sqrt(std::max(hh[0], 0.0));
      const double hnext = hcol[j + 1];   // zero: the Krylov space holds the solution
      ++it;
      if (hnext > 0.0) {
        note_launch();
        scale_into<<<G, 256, 0, s>>>(Vn, H->w, 1.0 / hcol[j + 1], nu);
      }
      // Givens rotations: apply the previous ones to the new column, then make a new one
      for (int i = 0; i < j; ++i) {
        const double a = hcol[i], b = hcol[i + 1];
        hcol[i] = cs_[i] * a + sn[i] * b;
        hcol[i + 1] = -sn[i] * a + cs_[i] * b;
      }
      const double den = std::hypot(hcol[j], hcol[j + 1]);
      cs_[j] = den > 0.0 ? hcol[j] / den : 1.0;
      sn[j] = den > 0.0 ? hcol[j + 1] / den : 0.0;
      hcol[j] = den;
      hcol[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs_[j] * g[j];
      for (int i = 0; i <= j; ++i) Hm[(size_t)i * m + j] = hcol[i];
      if (std::fabs(g[j + 1]) <= 0.5 * o->rtol * bnorm || hnext == 0.0) {
        ++j;
        break;
      }
    }
    // y = R^-1 g (back substitution), u += Z y
    for (int i = j - 1; i >= 0; --i) {
      double v = g[i];
      for (int k = i + 1; k < j; ++k) v -= Hm[(size_t)i * m + k] * y[k];
      y[i] = v / Hm[(size_t)i * m + i];
    }
    for (int i = 0; i < j; ++i) {
      note_launch();
      axpy_kernel<<<G, 256, 0, s>>>(u, H->Z + (size_t)i * nu, y[i], nu);
    }
  }
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(e, "dgw_helmholtz_solve");
  cudaEventRecord(H->ev_out, s);
  cudaStreamWaitEvent(cs, H->ev_out, 0);
  info->iterations = it;
  info->rel_residual = rel;
  info->ms = (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  info->dof_applies = (double)(dof_counter() - dof0);
  if (st == DGW_ENOTCONV) return set_error(DGW_ENOTCONV, "dgw_helmholtz_solve: max_iter reached");
  return DGW_OK;
}

}  // namespace dgw

namespace dgw {
// x = M^-1 r in every cell without switched-on enrichment (S^-1 W^-1 S^-T, exact there); cells with
// the wall model on get the block-diagonal approximation (the caller overwrites them)
cudaError_t launch_collocation_inverse_mass(dgw_mesh *M, const double *r, double *x, cudaStream_t s) {
  cudaError_t e = helm_setup(M, M->helm ? M->helm->m : 1);
  if (e != cudaSuccess) return e;
  return launch_inverse_mass(M, r, x, 1.0, s);
}
}  // namespace dgw

void dgw_helm_free(dgw_mesh *M) {
  if (!M || !M->helm) return;
  dgw::helm_free(M->helm);
  M->helm = nullptr;
}

using namespace dgw;

extern "C" dgw_status dgw_apply_mass(dgw_mesh_t M, int prec, const void *u, void *y, void *stream) {
  if (!M || !u || !y) return set_error(DGW_EINVAL, "dgw_apply_mass: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == DGW_FP64)
    return cuda_check(launch_vector_op<double>(OP_MASS, M->v64, (const double *)u, (double *)y, s), "dgw_apply_mass");
  if (prec == DGW_FP32) {
    if (!M->has32) return set_error(DGW_EINVAL, "dgw_apply_mass: mesh built without FP32 tables");
    return cuda_check(launch_vector_op<float>(OP_MASS, M->v32, (const float *)u, (float *)y, s), "dgw_apply_mass");
  }
  return set_error(DGW_EINVAL, "dgw_apply_mass: prec must be DGW_FP64 or DGW_FP32");
}

extern "C" dgw_status dgw_helmholtz_solve(dgw_mesh_t M, double gamma, const double *rhs, double *u,
                                          const dgw_helmholtz_opts *opts, dgw_solve_info *info, void *stream) {
  if (!M || !rhs || !u || !opts || !info) return set_error(DGW_EINVAL, "dgw_helmholtz_solve: null argument");
  if (!(gamma > 0) || !(opts->rtol > 0) || opts->max_iter < 1 || opts->restart < 0 || opts->restart > kMaxRestart)
    return set_error(DGW_EINVAL, "dgw_helmholtz_solve: gamma > 0, rtol > 0, max_iter >= 1, 0 <= restart <= 64");
  return helmholtz_solve(M, gamma, rhs, u, opts, info, (cudaStream_t)stream);
}
