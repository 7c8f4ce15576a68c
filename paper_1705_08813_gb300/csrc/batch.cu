// Mixed-precision pressure solves of several right-hand sides on one mesh at once (the request
// loop's continuous batching, and dgw_pressure_solve_batch).
//
// Every column is the solve of dgw_pressure_solve with mode 1 (Sec. 4.1 eq. poisson on the
// zero-mean subspace): FP64 iterative refinement (p, b - A p and its norm in FP64) around an FP32
// flexible CG with the FP32 multigrid V-cycle as preconditioner, each inner solve reducing the unit
// residual by max(1e-5, rtol ||b|| / (2 ||r||)). The columns share the launches: one FP32 operator
// launch, one V-cycle graph and one FP64 operator launch serve all of them (gridDim.y = column), and
// every reduction keeps per-column partial sums in a fixed order, so a column's arithmetic does not
// depend on which other columns run beside it.
//
// The batch advances in refinement rounds. A round computes the FP64 residual norm of every column,
// retires the converged ones, runs one inner solve for the others (columns whose inner solve has
// converged stop updating while the rest continue) and applies the refinement. Columns join and
// leave only between rounds; the caller compacts the block so the active columns are 0..ncols-1.
#include <algorithm>
#include <cstdint>
#include <type_traits>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "solver.h"

namespace dgw {

namespace {

constexpr int BR = 152;   // reduction blocks per column
enum { BS_RN = 0, BS_RZ, BS_RZNEW, BS_RZOLD, BS_DQ, BS_RR, BS_SUM, BS_BB, BS_COUNT = 8 };

inline int bgrid(long n) {
  long g = (n + 255) / 256;
  return (int)std::min<long>(std::max<long>(g, 1), 152 * 4);
}

template <typename T>
__device__ double bblock_sum(double v) {
  __shared__ double wp[32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wp[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? wp[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  }
  return s;
}

__device__ __forceinline__ bool baligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
__device__ __forceinline__ float bdot4(float4 x, float4 y) {
  return fmaf(x.w, y.w, fmaf(x.z, y.z, fmaf(x.y, y.y, x.x * y.x)));
}

// per column (blockIdx.y): partial[col][blockIdx.x] = sum a b (b null: sum a), FP64 accumulation (FP32
// columns: 16-byte loads, groups of four products summed in FP32 first)
template <typename T>
__global__ void bdot_partial(const T *__restrict__ a, const T *__restrict__ b, long n, double *__restrict__ partial) {
  const size_t co = (size_t)blockIdx.y * n;
  a += co;
  if (b) b += co;
  double s = 0.0;
  const long gid = blockIdx.x * (long)blockDim.x + threadIdx.x, stride = (long)gridDim.x * blockDim.x;
  long i0 = 0;
  if constexpr (std::is_same<T, float>::value) {
    if (baligned16(a) && (!b || baligned16(b))) {
      const long n4 = n >> 2;
      const float4 *a4 = reinterpret_cast<const float4 *>(a), *b4 = reinterpret_cast<const float4 *>(b);
      for (long i = gid; i < n4; i += stride) {
        const float4 x = a4[i];
        s += (double)(b ? bdot4(x, b4[i]) : (x.x + x.y) + (x.z + x.w));
      }
      i0 = n4 << 2;
    }
  }
  for (long i = i0 + gid; i < n; i += stride) s += b ? (double)a[i] * (double)b[i] : (double)a[i];
  s = bblock_sum<T>(s);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// one warp per column (blockIdx.x): sc[col][slot] = sum of the column's partials, fixed order
__global__ void bdot_finish(const double *__restrict__ partial, int np, double *__restrict__ sc, int slot) {
  const double *pc = partial + (size_t)blockIdx.x * np;
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += 32) s += pc[i];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (threadIdx.x == 0) sc[(size_t)blockIdx.x * BS_COUNT + slot] = s;
}

template <typename T>
void breduce(const T *a, const T *b, long n, int ncols, double *partial, double *sc, int slot, cudaStream_t s) {
  note_launches(2);
  bdot_partial<T><<<dim3(BR, ncols), 256, 0, s>>>(a, b, n, partial);
  bdot_finish<<<ncols, 32, 0, s>>>(partial, BR, sc, slot);
}

// x_col = a_col - sum_col / n (sum in sc[col][slot])
template <typename T>
__global__ void bsub_mean(const T *__restrict__ a, T *__restrict__ x, long n, const double *__restrict__ sc, int slot) {
  const size_t co = (size_t)blockIdx.y * n;
  const double m = sc[(size_t)blockIdx.y * BS_COUNT + slot] / (double)n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    x[co + i] = (T)((double)a[co + i] - m);
}

// r32 = r64 / ||r64|| per column
__global__ void bto_unit32(float *__restrict__ r32, const double *__restrict__ r, long n, const double *__restrict__ sc) {
  const size_t co = (size_t)blockIdx.y * n;
  const double s = 1.0 / sqrt(sc[(size_t)blockIdx.y * BS_COUNT + BS_RN]);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    r32[co + i] = (float)(r[co + i] * s);
}

// e += alpha d, r -= alpha q (alpha = rz / dq) for the columns whose inner solve still runs and, in the
// same pass, the partial sums of r.r (partial[col][blk]) and of r.z (partial[ncols + col][blk]) of the
// updated r and z, which still holds the previous preconditioned residual (the r.z_old of the
// flexible beta); columns that have stopped write zeros.
__global__ void bpcg_update_dots(float *__restrict__ e, float *__restrict__ r, const float *__restrict__ d,
                                 const float *__restrict__ q, const float *__restrict__ z, long n,
                                 const double *__restrict__ sc, const int *__restrict__ run, double *__restrict__ partial) {
  const int col = blockIdx.y, ncols = gridDim.y;
  double srr = 0.0, srz = 0.0;
  if (run[col]) {
    const size_t co = (size_t)col * n;
    e += co; r += co; d += co; q += co; z += co;
    const double *c = sc + (size_t)col * BS_COUNT;
    const float alpha = (float)(c[BS_RZ] / c[BS_DQ]);
    const long gid = blockIdx.x * (long)blockDim.x + threadIdx.x, stride = (long)gridDim.x * blockDim.x;
    long i0 = 0;
    if (baligned16(e) && baligned16(r) && baligned16(d) && baligned16(q) && baligned16(z)) {
      const long n4 = n >> 2;
      float4 *e4 = reinterpret_cast<float4 *>(e), *r4 = reinterpret_cast<float4 *>(r);
      const float4 *d4 = reinterpret_cast<const float4 *>(d), *q4 = reinterpret_cast<const float4 *>(q);
      const float4 *z4 = reinterpret_cast<const float4 *>(z);
      for (long i = gid; i < n4; i += stride) {
        float4 ev = e4[i], rv = r4[i];
        const float4 dv = d4[i], qv = q4[i], zv = z4[i];
        ev.x += alpha * dv.x; ev.y += alpha * dv.y; ev.z += alpha * dv.z; ev.w += alpha * dv.w;
        rv.x -= alpha * qv.x; rv.y -= alpha * qv.y; rv.z -= alpha * qv.z; rv.w -= alpha * qv.w;
        e4[i] = ev;
        r4[i] = rv;
        srr += (double)bdot4(rv, rv);
        srz += (double)bdot4(rv, zv);
      }
      i0 = n4 << 2;
    }
    for (long i = i0 + gid; i < n; i += stride) {
      e[i] += alpha * d[i];
      const float rn = r[i] - alpha * q[i];
      r[i] = rn;
      srr += (double)rn * (double)rn;
      srz += (double)rn * (double)z[i];
    }
  }
  srr = bblock_sum<float>(srr);
  srz = bblock_sum<float>(srz);
  if (threadIdx.x == 0) {
    partial[(size_t)col * gridDim.x + blockIdx.x] = srr;
    partial[(size_t)(ncols + col) * gridDim.x + blockIdx.x] = srz;
  }
}

// d = z (first) or z + beta d with the flexible beta = (r.z - r.z_old) / rz_old, then rz <- rz_new
__global__ void bpcg_direction(float *__restrict__ d, const float *__restrict__ z, long n, const double *__restrict__ sc,
                               int first, const int *__restrict__ run) {
  if (!run[blockIdx.y]) return;
  const size_t co = (size_t)blockIdx.y * n;
  const double *c = sc + (size_t)blockIdx.y * BS_COUNT;
  const float beta = first ? 0.0f : (float)((c[BS_RZNEW] - c[BS_RZOLD]) / c[BS_RZ]);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    d[co + i] = first ? z[co + i] : z[co + i] + beta * d[co + i];
}

__global__ void bshift_rz(double *sc, int ncols, const int *__restrict__ run) {
  const int c = threadIdx.x;
  if (c < ncols && run[c]) sc[(size_t)c * BS_COUNT + BS_RZ] = sc[(size_t)c * BS_COUNT + BS_RZNEW];
}

// z32 -= mean(z32) per column (the V-cycle output on the zero-mean subspace)
__global__ void bsub_mean32(float *__restrict__ z, long n, const double *__restrict__ sc) {
  const size_t co = (size_t)blockIdx.y * n;
  const float m = (float)(sc[(size_t)blockIdx.y * BS_COUNT + BS_SUM] / (double)n);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) z[co + i] -= m;
}

// p += ||r|| e, the scaled correction of the unit right-hand side
__global__ void baccumulate(double *__restrict__ p, const float *__restrict__ e, long n, const double *__restrict__ sc) {
  const size_t co = (size_t)blockIdx.y * n;
  const double s = sqrt(sc[(size_t)blockIdx.y * BS_COUNT + BS_RN]);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    p[co + i] += s * (double)e[co + i];
}

// r = b - q over a block of columns
__global__ void bresidual(double *__restrict__ r, const double *__restrict__ b, const double *__restrict__ q, long n) {
  const size_t co = (size_t)blockIdx.y * n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    r[co + i] = b[co + i] - q[co + i];
}

}  // namespace

struct Batch {
  dgw_mesh *M = nullptr;
  int cap = 0;
  long n = 0;
  cudaStream_t stream = nullptr;
  void *mg = nullptr;
  int cheb = 5;
  float *r32 = nullptr, *z32 = nullptr;   // the hierarchy's level-0 blocks
  float *d32 = nullptr, *q32 = nullptr, *e32 = nullptr;
  double *b64 = nullptr, *r64 = nullptr, *p64 = nullptr, *q64 = nullptr;
  double *partial = nullptr, *sc = nullptr, *host_sc = nullptr;
  int *run = nullptr, *host_run = nullptr;
  std::vector<cudaGraphExec_t> graphs;    // V-cycle + mean projection per column count
  std::vector<unsigned long long> graph_launches, graph_dofs;
  std::vector<void *> allocs;
  std::vector<BatchColumn> col;           // host state per column
};

namespace {

template <typename T>
T *balloc(Batch *B, size_t n, cudaError_t &e) {
  void *p = nullptr;
  if (e != cudaSuccess) return nullptr;
  e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
  if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, std::max<size_t>(n, 1) * sizeof(T), B->stream);
  if (e == cudaSuccess) B->allocs.push_back(p);
  return static_cast<T *>(p);
}

// one V-cycle over the first ncols columns of r32 -> z32 and the zero-mean projection of z32, as a
// CUDA graph captured on first use per column count
cudaError_t vcycle_block(Batch *B, int ncols) {
  cudaStream_t s = B->stream;
  if (!B->graphs[ncols]) {
    const unsigned long long l0 = launch_counter(), d0 = dof_counter();
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t ev = mg_batch_vcycle(B->mg, ncols, s);
    if (ev == cudaSuccess) {
      breduce<float>(B->z32, nullptr, B->n, ncols, B->partial, B->sc, BS_SUM, s);
      note_launch();
      bsub_mean32<<<dim3(bgrid(B->n), ncols), 256, 0, s>>>(B->z32, B->n, B->sc);
      ev = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (ev != cudaSuccess) e = ev;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&B->graphs[ncols], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) { B->graphs[ncols] = nullptr; return e; }
    B->graph_launches[ncols] = launch_counter() - l0;
    B->graph_dofs[ncols] = dof_counter() - d0;
    return cudaGraphLaunch(B->graphs[ncols], s);
  }
  note_launches(B->graph_launches[ncols]);
  note_dofs((long long)B->graph_dofs[ncols]);
  return cudaGraphLaunch(B->graphs[ncols], s);
}

cudaError_t sync_scalars(Batch *B, int ncols) {
  cudaError_t e = cudaMemcpyAsync(B->host_sc, B->sc, (size_t)ncols * BS_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                                  B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  return e;
}

cudaError_t upload_run(Batch *B, int ncols) {
  return cudaMemcpyAsync(B->run, B->host_run, ncols * sizeof(int), cudaMemcpyHostToDevice, B->stream);
}

}  // namespace

void batch_destroy(Batch *B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream);
  for (auto g : B->graphs)
    if (g) cudaGraphExecDestroy(g);
  if (B->mg) mg_batch_free(B->mg);
  for (void *p : B->allocs) cudaFree(p);
  if (B->host_sc) cudaFreeHost(B->host_sc);
  if (B->host_run) cudaFreeHost(B->host_run);
  if (B->stream) cudaStreamDestroy(B->stream);
  delete B;
}

cudaError_t batch_create(dgw_mesh *M, int cap, int cheb, Batch **out) {
  *out = nullptr;
  if (M->P.geometry != 0 || !M->has32 || cap < 1 || cap > kBatchMax) return cudaErrorNotSupported;
  Batch *B = new Batch();
  B->M = M;
  B->cap = cap;
  B->n = M->np;
  B->cheb = cheb;
  cudaError_t e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = mg_batch_create(M, cap, cheb, B->stream, &B->mg);
  if (e == cudaSuccess) mg_batch_level0(B->mg, &B->r32, &B->z32);
  const size_t nb = (size_t)B->n * cap;
  B->d32 = balloc<float>(B, nb, e);
  B->q32 = balloc<float>(B, nb, e);
  B->e32 = balloc<float>(B, nb, e);
  B->b64 = balloc<double>(B, nb, e);
  B->r64 = balloc<double>(B, nb, e);
  B->p64 = balloc<double>(B, nb, e);
  B->q64 = balloc<double>(B, nb, e);
  B->partial = balloc<double>(B, (size_t)2 * BR * cap, e);   // two partial sums per column (update + dots)
  B->sc = balloc<double>(B, (size_t)BS_COUNT * cap, e);
  B->run = balloc<int>(B, cap, e);
  if (e == cudaSuccess) e = cudaMallocHost(&B->host_sc, (size_t)BS_COUNT * cap * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&B->host_run, cap * sizeof(int));
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  B->graphs.assign(cap + 1, nullptr);
  B->graph_launches.assign(cap + 1, 0);
  B->graph_dofs.assign(cap + 1, 0);
  B->col.assign(cap, BatchColumn{});
  if (e != cudaSuccess) {
    batch_destroy(B);
    return e;
  }
  *out = B;
  return cudaSuccess;
}

int batch_active(const Batch *B) {
  int k = 0;
  while (k < B->cap && B->col[k].used) ++k;
  return k;
}

// Column slot batch_active(B) takes the right-hand side b_in (projected to zero mean), p = 0.
cudaError_t batch_admit(Batch *B, const BatchColumn &c, cudaStream_t caller) {
  const int k = batch_active(B);
  if (k >= B->cap) return cudaErrorInvalidValue;
  cudaStream_t s = B->stream;
  cudaEvent_t ev = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, caller);   // b_in is written on the caller's stream
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
  if (ev) cudaEventDestroy(ev);
  const long n = B->n;
  const size_t co = (size_t)k * n;
  // b = b_in - mean(b_in) in column k; ||b||; r = b; p = 0
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->b64 + co, c.b_in, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  breduce<double>(B->b64 + co, nullptr, n, 1, B->partial, B->sc, BS_SUM, s);
  note_launch();
  bsub_mean<double><<<bgrid(n), 256, 0, s>>>(B->b64 + co, B->b64 + co, n, B->sc, BS_SUM);
  breduce<double>(B->b64 + co, B->b64 + co, n, 1, B->partial, B->sc, BS_BB, s);
  e = cudaMemcpyAsync(B->r64 + co, B->b64 + co, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(B->p64 + co, 0, n * sizeof(double), s);
  if (e == cudaSuccess) e = sync_scalars(B, 1);
  if (e != cudaSuccess) return e;
  B->col[k] = c;
  B->col[k].used = true;
  B->col[k].bnorm = std::sqrt(std::max(B->host_sc[BS_BB], 0.0));
  B->col[k].iterations = 0;
  B->col[k].t_admit = std::chrono::steady_clock::now();
  return cudaSuccess;
}

// Move column src into slot dst (both below the active count; dst is finished).
static cudaError_t batch_move(Batch *B, int src, int dst) {
  const long n = B->n;
  cudaStream_t s = B->stream;
  cudaError_t e = cudaSuccess;
  for (double *v : {B->b64, B->r64, B->p64})
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(v + (size_t)dst * n, v + (size_t)src * n, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  B->col[dst] = B->col[src];
  B->col[src] = BatchColumn{};
  return e;
}

// One refinement round over the active columns 0..ncols-1; finished columns (converged, failed to
// converge within max_iter, or with a zero right-hand side) get their result written to p_out and
// are appended to done, and the block is compacted.
cudaError_t batch_round(Batch *B, std::vector<BatchColumn> &done) {
  cudaStream_t s = B->stream;
  const long n = B->n;
  int ncols = batch_active(B);
  if (ncols == 0) return cudaSuccess;
  const int G = bgrid(n);
  // FP64 residual norms
  breduce<double>(B->r64, B->r64, n, ncols, B->partial, B->sc, BS_RN, s);
  cudaError_t e = sync_scalars(B, ncols);
  if (e != cudaSuccess) return e;
  std::vector<double> tol_in(ncols, 0.0);
  bool any_finished = false;
  for (int c = 0; c < ncols; ++c) {
    BatchColumn &C = B->col[c];
    const double rn = std::sqrt(std::max(B->host_sc[(size_t)c * BS_COUNT + BS_RN], 0.0));
    C.rel_residual = C.bnorm > 0.0 ? rn / C.bnorm : 0.0;
    if (C.bnorm == 0.0 || rn <= C.rtol * C.bnorm) { C.status = DGW_OK; C.finished = true; }
    else if (C.iterations >= C.max_iter) { C.status = DGW_ENOTCONV; C.finished = true; }
    else tol_in[c] = std::max(1e-5, 0.5 * C.rtol * C.bnorm / rn);
    any_finished = any_finished || C.finished;
  }
  if (any_finished) {
    // results: p - mean(p) into the caller's buffer (the residual norm is unchanged by the shift)
    for (int c = 0; c < ncols; ++c) {
      BatchColumn &C = B->col[c];
      if (!C.finished) continue;
      const size_t co = (size_t)c * n;
      breduce<double>(B->p64 + co, nullptr, n, 1, B->partial, B->sc, BS_SUM, s);
      note_launch();
      bsub_mean<double><<<G, 256, 0, s>>>(B->p64 + co, C.p_out, n, B->sc, BS_SUM);
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    // compaction: the unfinished columns move, in order, into slots 0..kept-1
    std::vector<int> keep;
    for (int c = 0; c < ncols; ++c) {
      if (B->col[c].finished) {
        done.push_back(B->col[c]);
        B->col[c] = BatchColumn{};
      } else {
        keep.push_back(c);
      }
    }
    for (int i = 0; i < (int)keep.size(); ++i) {
      if (keep[i] == i) continue;
      e = batch_move(B, keep[i], i);   // slot i is free: keep is increasing
      if (e != cudaSuccess) return e;
      tol_in[i] = tol_in[keep[i]];
    }
    ncols = batch_active(B);
    if (ncols == 0) return cudaSuccess;
    breduce<double>(B->r64, B->r64, n, ncols, B->partial, B->sc, BS_RN, s);   // norms of the moved columns
  }
  // one inner FP32 solve per active column
  for (int c = 0; c < ncols; ++c) B->host_run[c] = 1;
  e = upload_run(B, ncols);
  if (e != cudaSuccess) return e;
  note_launch();
  bto_unit32<<<dim3(G, ncols), 256, 0, s>>>(B->r32, B->r64, n, B->sc);
  e = cudaMemsetAsync(B->e32, 0, (size_t)ncols * n * sizeof(float), s);
  if (e == cudaSuccess) e = vcycle_block(B, ncols);
  if (e != cudaSuccess) return e;
  breduce<float>(B->r32, B->z32, n, ncols, B->partial, B->sc, BS_RZNEW, s);
  note_launches(2);
  bpcg_direction<<<dim3(G, ncols), 256, 0, s>>>(B->d32, B->z32, n, B->sc, 1, B->run);
  bshift_rz<<<1, 32, 0, s>>>(B->sc, ncols, B->run);
  LapEpi<float> e32{};
  e32.mode = LAP_PLAIN;
  e32.ncols = ncols;
  for (;;) {
    e = launch_laplace_epi<float>(B->M->v32, B->d32, B->q32, e32, s);
    if (e != cudaSuccess) return e;
    breduce<float>(B->d32, B->q32, n, ncols, B->partial, B->sc, BS_DQ, s);
    // the update with r.r and r.z_old (z32 still holds the previous preconditioned residuals)
    note_launches(3);
    bpcg_update_dots<<<dim3(BR, ncols), 256, 0, s>>>(B->e32, B->r32, B->d32, B->q32, B->z32, n, B->sc, B->run,
                                                     B->partial);
    bdot_finish<<<ncols, 32, 0, s>>>(B->partial, BR, B->sc, BS_RR);
    bdot_finish<<<ncols, 32, 0, s>>>(B->partial + (size_t)ncols * BR, BR, B->sc, BS_RZOLD);
    e = sync_scalars(B, ncols);
    if (e != cudaSuccess) return e;
    bool any = false;
    for (int c = 0; c < ncols; ++c) {
      if (!B->host_run[c]) continue;
      BatchColumn &C = B->col[c];
      ++C.iterations;
      const double rr = std::sqrt(std::max(B->host_sc[(size_t)c * BS_COUNT + BS_RR], 0.0));
      if (rr <= tol_in[c] || C.iterations >= C.max_iter) B->host_run[c] = 0;
      any = any || B->host_run[c];
    }
    if (!any) break;
    e = upload_run(B, ncols);
    if (e == cudaSuccess) e = vcycle_block(B, ncols);
    if (e != cudaSuccess) return e;
    breduce<float>(B->r32, B->z32, n, ncols, B->partial, B->sc, BS_RZNEW, s);
    note_launches(2);
    bpcg_direction<<<dim3(G, ncols), 256, 0, s>>>(B->d32, B->z32, n, B->sc, 0, B->run);
    bshift_rz<<<1, 32, 0, s>>>(B->sc, ncols, B->run);
  }
  // refinement: p += ||r|| e; r = b - A p in FP64
  note_launch();
  baccumulate<<<dim3(G, ncols), 256, 0, s>>>(B->p64, B->e32, n, B->sc);
  LapEpi<double> e64{};
  e64.mode = LAP_PLAIN;
  e64.ncols = ncols;
  e = launch_laplace_epi<double>(B->M->v64, B->p64, B->q64, e64, s);
  if (e != cudaSuccess) return e;
  note_launch();
  bresidual<<<dim3(G, ncols), 256, 0, s>>>(B->r64, B->b64, B->q64, n);
  return cudaGetLastError();
}

}  // namespace dgw

void dgw_batch_free(dgw_mesh *M) {
  if (M && M->batch) {
    dgw::batch_destroy(M->batch);
    M->batch = nullptr;
  }
}

extern "C" dgw_status dgw_pressure_solve_batch(dgw_mesh_t M, int ncols, const double *const *b, double *const *p,
                                               const dgw_solve_opts *opts, dgw_solve_info *infos, void *stream) {
  using namespace dgw;
  if (!M || !b || !p || !opts || !infos || ncols < 1)
    return set_error(DGW_EINVAL, "dgw_pressure_solve_batch: null argument or ncols < 1");
  for (int c = 0; c < ncols; ++c)
    if (!b[c] || !p[c]) return set_error(DGW_EINVAL, "dgw_pressure_solve_batch: null column pointer");
  if (!(opts->rtol > 0) || opts->max_iter < 1 || opts->mode != 1)
    return set_error(DGW_EINVAL, "dgw_pressure_solve_batch: rtol > 0, max_iter >= 1 and mode 1 required");
  if (M->P.geometry != 0 || !M->has32)
    return set_error(DGW_EINVAL, "dgw_pressure_solve_batch: needs box cells (geometry 0) with FP32 tables");
  const int cheb = opts->cheb_degree > 0 ? opts->cheb_degree : 5;
  if (M->batch && M->batch_cheb != cheb) dgw_batch_free(M);
  if (!M->batch) {
    Batch *B = nullptr;
    const cudaError_t e = batch_create(M, kBatchMax, cheb, &B);
    if (e == cudaErrorNotSupported)
      return set_error(DGW_EINVAL, "dgw_pressure_solve_batch: the mesh's multigrid hierarchy needs the iterative coarse solve");
    if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve_batch: batch workspace");
    M->batch = B;
    M->batch_cheb = cheb;
  }
  Batch *B = M->batch;
  const unsigned long long dof0 = dof_counter();
  int next = 0, left = ncols;
  std::vector<BatchColumn> done;
  while (left > 0) {
    while (next < ncols && batch_active(B) < B->cap) {   // admit as columns free up
      BatchColumn c;
      c.b_in = b[next];
      c.p_out = p[next];
      c.tag = next;
      c.caller_stream = stream;
      c.rtol = opts->rtol;
      c.max_iter = opts->max_iter;
      const cudaError_t e = batch_admit(B, c, (cudaStream_t)stream);
      if (e != cudaSuccess) {
        dgw_batch_free(M);   // the block holds this call's columns: the next call starts from a new one
        return cuda_check(e, "dgw_pressure_solve_batch: admission");
      }
      ++next;
    }
    done.clear();
    const cudaError_t e = batch_round(B, done);
    if (e != cudaSuccess) {
      dgw_batch_free(M);
      return cuda_check(e, "dgw_pressure_solve_batch");
    }
    for (const BatchColumn &c : done) {
      dgw_solve_info &inf = infos[c.tag];
      inf.iterations = c.iterations;
      inf.rel_residual = c.rel_residual;
      inf.ms = (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - c.t_admit).count();
      inf.dof_applies = 0.0;
      --left;
    }
  }
  const double dofs = (double)(dof_counter() - dof0);
  dgw_status st = DGW_OK;
  for (int c = 0; c < ncols; ++c) {
    infos[c].dof_applies = dofs / ncols;
    if (infos[c].rel_residual > opts->rtol) st = DGW_ENOTCONV;
  }
  if (st == DGW_ENOTCONV) return set_error(DGW_ENOTCONV, "dgw_pressure_solve_batch: max_iter reached in a column");
  return DGW_OK;
}
