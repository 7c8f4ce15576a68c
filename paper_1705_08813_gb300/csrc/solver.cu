// Pressure Poisson solve: preconditioned CG on -L p = b restricted to zero-mean vectors
// (Sec. 4.1 eq. poisson, Sec. 4.2 eq. poissonspat; the null space of the pure-Neumann/periodic
// SIPG operator is the constant vector). Deterministic two-stage reductions; FP64 vectors,
// residuals and dot products.
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <string>
#include <vector>

#include "dgw_internal.h"
#include "solver.h"

namespace dgw {

constexpr int RED_THREADS = 256;

// Block-level sum for a fixed-order reduction.
template <typename T>
__device__ T block_sum(T v) {
  __shared__ T warp_part[32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) warp_part[w] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? warp_part[threadIdx.x] : T(0);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  }
  __syncthreads();
  return s;
}

// partial[blockIdx] = sum_i a_i b_i (b == nullptr: sum_i a_i)
__global__ void dot_partial_kernel(const double *__restrict__ a, const double *__restrict__ b, long n,
                                   double *__restrict__ partial) {
  double s = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    s += b ? a[i] * b[i] : a[i];
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out[slot] = sum of partials (one warp, fixed order)
__global__ void dot_finish_kernel(const double *__restrict__ partial, int np, double *__restrict__ out, int slot) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += 32) s += partial[i];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (threadIdx.x == 0) out[slot] = s;
}

// x = a - mean(a) where the sum of a is sc[slot]
__global__ void sub_mean_kernel(const double *__restrict__ a, double *__restrict__ x, long n, const double *sc,
                                int slot) {
  const double m = sc[slot] / (double)n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) x[i] = a[i] - m;
}

// p += alpha d; r -= alpha q with alpha = sc[RZ] / sc[DQ]
__global__ void cg_update_kernel(double *__restrict__ p, double *__restrict__ r, const double *__restrict__ d,
                                 const double *__restrict__ q, long n, const double *sc) {
  const double alpha = sc[SC_RZ] / sc[SC_DQ];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    p[i] += alpha * d[i];
    r[i] -= alpha * q[i];
  }
}

// z = r / diag
__global__ void jacobi_kernel(const double *__restrict__ r, const double *__restrict__ dg, double *__restrict__ z,
                              long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    z[i] = r[i] / dg[i];
}

// d = z + beta d with the flexible (Polak-Ribiere) beta = (r.z - r.z_old) / rz_old, which
// equals the standard beta for a fixed linear preconditioner and stays robust when the
// preconditioner varies slightly between iterations (FP32 multigrid, inner coarse PCG).
// sc[RZ] = sc[RZNEW] is shifted by a separate launch.
__global__ void cg_direction_kernel(double *__restrict__ d, const double *__restrict__ z, long n, const double *sc,
                                    int first) {
  const double beta = first ? 0.0 : (sc[SC_RZNEW] - sc[SC_RZOLD]) / sc[SC_RZ];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    d[i] = first ? z[i] : z[i] + beta * d[i];   // d is not read on the first step (may be uninitialised)
}

__global__ void copy_scalar_kernel(double *sc, int dst, int src) {
  if (threadIdx.x == 0 && blockIdx.x == 0) sc[dst] = sc[src];
}

__global__ void axpby_kernel(double *__restrict__ y, const double *__restrict__ x, double a, double b, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

// ---- FP32 vectors of the mixed-precision inner solve (reductions accumulate in FP64)

__device__ __forceinline__ bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// x . y of four FP32 pairs in FP32 (the group sum then goes into an FP64 accumulator)
__device__ __forceinline__ float dot4(float4 x, float4 y) {
  return fmaf(x.w, y.w, fmaf(x.z, y.z, fmaf(x.y, y.y, x.x * y.x)));
}

// partial[blockIdx] = sum_i a_i b_i (b == nullptr: sum_i a_i), FP32 inputs: 16-byte loads, each group
// of four products summed in FP32 and accumulated in FP64 (the FP64 units of this part do a quarter
// of the work of a per-element FP64 accumulation); fixed order for a given launch shape.
__global__ void dot32_partial_kernel(const float *__restrict__ a, const float *__restrict__ b, long n,
                                     double *__restrict__ partial) {
  double s = 0.0;
  const long gid = blockIdx.x * (long)blockDim.x + threadIdx.x, stride = (long)gridDim.x * blockDim.x;
  long i0 = 0;
  if (aligned16(a) && (!b || aligned16(b))) {
    const long n4 = n >> 2;
    const float4 *a4 = reinterpret_cast<const float4 *>(a), *b4 = reinterpret_cast<const float4 *>(b);
    for (long i = gid; i < n4; i += stride) {
      const float4 x = a4[i];
      s += (double)(b ? dot4(x, b4[i]) : (x.x + x.y) + (x.z + x.w));
    }
    i0 = n4 << 2;
  }
  for (long i = i0 + gid; i < n; i += stride) s += b ? (double)a[i] * (double)b[i] : (double)a[i];
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// r32 = r / sqrt(sc[slot]) (the outer residual normalised to unit 2-norm)
__global__ void to_unit32_kernel(float *__restrict__ r32, const double *__restrict__ r, long n, const double *sc,
                                 int slot) {
  const double s = 1.0 / sqrt(sc[slot]);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    r32[i] = (float)(r[i] * s);
}


// e += alpha d, r -= alpha q (alpha = sc[RZ] / sc[DQ]) and, in the same pass, the partial sums of
// r.r (partial[blk]) and r.z (partial[RED_BLOCKS + blk]) of the updated r with z, which still holds
// the previous preconditioned residual (the r.z_old of the flexible beta)
__global__ void pcg32_update_dots_kernel(float *__restrict__ e, float *__restrict__ r, const float *__restrict__ d,
                                         const float *__restrict__ q, const float *__restrict__ z, long n,
                                         const double *sc, double *__restrict__ partial) {
  const float alpha = (float)(sc[SC_RZ] / sc[SC_DQ]);
  double srr = 0.0, srz = 0.0;
  const long gid = blockIdx.x * (long)blockDim.x + threadIdx.x, stride = (long)gridDim.x * blockDim.x;
  long i0 = 0;
  if (aligned16(e) && aligned16(r) && aligned16(d) && aligned16(q) && aligned16(z)) {
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
      srr += (double)dot4(rv, rv);
      srz += (double)dot4(rv, zv);
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
  srr = block_sum(srr);
  srz = block_sum(srz);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = srr;
    partial[RED_BLOCKS + blockIdx.x] = srz;
  }
}

// d = z (first) or z + beta d, flexible beta = (r.z - r.z_old) / rz_old
__global__ void pcg32_direction_kernel(float *__restrict__ d, const float *__restrict__ z, long n, const double *sc,
                                       int first) {
  const float beta = first ? 0.0f : (float)((sc[SC_RZNEW] - sc[SC_RZOLD]) / sc[SC_RZ]);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    d[i] = first ? z[i] : z[i] + beta * d[i];
}

// x -= mean(x), the sum of x in sc[slot]
__global__ void sub_mean32_kernel(float *__restrict__ x, long n, const double *sc, int slot) {
  const float m = (float)(sc[slot] / (double)n);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) x[i] -= m;
}

// p += sqrt(sc[slot]) e: the correction of the unit right-hand side scaled back
__global__ void accumulate64_kernel(double *__restrict__ p, const float *__restrict__ e, long n, const double *sc,
                                    int slot) {
  const double s = sqrt(sc[slot]);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    p[i] += s * (double)e[i];
}

static inline int grid_for(long n) {
  long g = (n + 255) / 256;
  return (int)std::min<long>(std::max<long>(g, 1), 152 * 16);
}

cudaError_t reduce_to(const double *a, const double *b, long n, double *partial, double *sc, int slot,
                      cudaStream_t s) {
  note_launch();
  dot_partial_kernel<<<RED_BLOCKS, RED_THREADS, 0, s>>>(a, b, n, partial);
  note_launch();
  dot_finish_kernel<<<1, 32, 0, s>>>(partial, RED_BLOCKS, sc, slot);
  return cudaGetLastError();
}

static cudaError_t reduce32_to(const float *a, const float *b, long n, double *partial, double *sc, int slot,
                               cudaStream_t s) {
  note_launch();
  dot32_partial_kernel<<<RED_BLOCKS, RED_THREADS, 0, s>>>(a, b, n, partial);
  note_launch();
  dot_finish_kernel<<<1, 32, 0, s>>>(partial, RED_BLOCKS, sc, slot);
  return cudaGetLastError();
}

cudaError_t project_mean(const double *a, double *x, long n, double *partial, double *sc, int slot, cudaStream_t s) {
  cudaError_t e = reduce_to(a, nullptr, n, partial, sc, slot, s);
  if (e != cudaSuccess) return e;
  note_launch();
  sub_mean_kernel<<<grid_for(n), 256, 0, s>>>(a, x, n, sc, slot);
  return cudaGetLastError();
}

dgw_solver *get_solver(dgw_mesh *M) {
  if (M->solver) return M->solver;
  dgw_solver *S = new dgw_solver();
  const long n = M->np;
  cudaError_t e = cudaSuccess;
  double **vecs[] = {&S->b, &S->r, &S->z, &S->d, &S->q, &S->zold, &S->partial, &S->sc};
  const size_t sizes[] = {(size_t)n, (size_t)n, (size_t)n, (size_t)n, (size_t)n, (size_t)n, (size_t)2 * RED_BLOCKS,
                          (size_t)SC_COUNT};
  e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  for (int i = 0; i < 8 && e == cudaSuccess; ++i) {
    e = cudaMalloc(vecs[i], sizes[i] * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(*vecs[i], 0, sizes[i] * sizeof(double), S->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
  if (e == cudaSuccess) e = cudaMallocHost(&S->host_sc, SC_COUNT * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&S->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&S->ev1);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_out, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    M->solver = S;
    dgw_solver_free(M);
    return nullptr;
  }
  M->solver = S;
  return S;
}

// The V-cycle r -> z as a CUDA graph: captured once per hierarchy on the internal stream and
// replayed every CG iteration (about 300 small launches per cycle otherwise).
static cudaError_t vcycle_graph(dgw_mesh *M, dgw_solver *S, int mode, cudaStream_t s) {
  if (S->vgraph) return cudaGraphLaunch(S->vgraph, s) == cudaSuccess
                             ? (note_launches(S->vgraph_launches), note_dofs((long long)S->vgraph_dofs), cudaSuccess)
                             : cudaErrorLaunchFailure;
  const unsigned long long l0 = launch_counter(), d0 = dof_counter();
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t ev = mg_vcycle(M, S, mode, S->r, S->z, s);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s, &g);
  if (ev != cudaSuccess) e = ev;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&S->vgraph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) { S->vgraph = nullptr; return e; }
  S->vgraph_launches = launch_counter() - l0;
  S->vgraph_dofs = dof_counter() - d0;
  // the capture itself counted nothing that ran; the launch below runs and counts it
  e = cudaGraphLaunch(S->vgraph, s);
  return e;
}

// One FP32 V-cycle on the finest level's buffers (r32 -> z32) followed by the projection of z32 onto
// zero mean, as a CUDA graph captured on first use per hierarchy and replayed every inner iteration.
static cudaError_t vcycle32_graph(dgw_mesh *M, dgw_solver *S, float *z32, cudaStream_t s) {
  const long n = M->np;
  const int G = grid_for(n);
  if (!S->vgraph32) {
    const unsigned long long l0 = launch_counter(), d0 = dof_counter();
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t ev = mg_vcycle_f32(S, s);
    if (ev == cudaSuccess) ev = reduce32_to(z32, nullptr, n, S->partial, S->sc, SC_TMP, s);
    if (ev == cudaSuccess) {
      note_launch();
      sub_mean32_kernel<<<G, 256, 0, s>>>(z32, n, S->sc, SC_TMP);
      ev = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (ev != cudaSuccess) e = ev;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&S->vgraph32, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) { S->vgraph32 = nullptr; return e; }
    // the capture counted the launches and DoFs of one replay: they stand for the launch below, and
    // every later replay adds them again
    S->vgraph32_launches = launch_counter() - l0;
    S->vgraph32_dofs = dof_counter() - d0;
    return cudaGraphLaunch(S->vgraph32, s);
  }
  note_launches(S->vgraph32_launches);
  note_dofs((long long)S->vgraph32_dofs);
  return cudaGraphLaunch(S->vgraph32, s);
}

// Mixed precision (mode 1): FP64 iterative refinement around an FP32 preconditioned CG. The outer
// loop keeps p, the residual r = b - A p and its norm in FP64 (one FP64 operator apply per outer
// step); each inner solve takes the residual scaled to unit norm, runs flexible CG with the FP32
// operator and the FP32 multigrid V-cycle (dot products accumulated in FP64) until the unit
// residual drops below max(1e-5, rtol ||b|| / (2 ||r||)), and the scaled correction is added to p.
static dgw_status pressure_solve_mixed(dgw_mesh *M, dgw_solver *S, const dgw_solve_opts *o, double *p, double bnorm,
                                       int *iterations, cudaStream_t s) {
  const long n = M->np;
  const int G = grid_for(n);
  float *r32 = nullptr, *z32 = nullptr;
  cudaError_t e = mg_level0_f32(S, &r32, &z32);
  if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve: mixed hierarchy");
  if (!S->d32) {
    float **v32[] = {&S->d32, &S->q32, &S->e32};
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
      e = cudaMalloc(v32[i], n * sizeof(float));
      if (e == cudaSuccess) e = cudaMemsetAsync(*v32[i], 0, n * sizeof(float), s);
    }
    if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve: mixed workspace");
  }
  constexpr double kInnerTol = 1e-5;   // reduction per inner solve; FP32 rounding allows about 1e-6
  int it = 0;
  for (;;) {
    // S->r holds the FP64 residual of p; its squared norm goes to SC_RN
    reduce_to(S->r, S->r, n, S->partial, S->sc, SC_RN, s);
    cudaMemcpyAsync(S->host_sc, S->sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve");
    const double rn = std::sqrt(std::max(S->host_sc[SC_RN], 0.0));
    if (rn <= o->rtol * bnorm) break;
    if (it >= o->max_iter) { *iterations = it; return DGW_ENOTCONV; }
    const double tol_in = std::max(kInnerTol, 0.5 * o->rtol * bnorm / rn);
    note_launch();
    to_unit32_kernel<<<G, 256, 0, s>>>(r32, S->r, n, S->sc, SC_RN);
    cudaMemsetAsync(S->e32, 0, n * sizeof(float), s);
    e = vcycle32_graph(M, S, z32, s);
    if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve: preconditioner");
    reduce32_to(r32, z32, n, S->partial, S->sc, SC_RZNEW, s);
    note_launch();
    pcg32_direction_kernel<<<G, 256, 0, s>>>(S->d32, z32, n, S->sc, 1);
    note_launch();
    copy_scalar_kernel<<<1, 1, 0, s>>>(S->sc, SC_RZ, SC_RZNEW);
    for (;;) {
      e = launch_laplace<float>(M->v32, S->d32, S->q32, s);
      if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve: operator");
      reduce32_to(S->d32, S->q32, n, S->partial, S->sc, SC_DQ, s);
      // the update with r.r and r.z_old (z32 still holds the previous preconditioned residual)
      note_launches(3);
      pcg32_update_dots_kernel<<<RED_BLOCKS, RED_THREADS, 0, s>>>(S->e32, r32, S->d32, S->q32, z32, n, S->sc, S->partial);
      dot_finish_kernel<<<1, 32, 0, s>>>(S->partial, RED_BLOCKS, S->sc, SC_RR);
      dot_finish_kernel<<<1, 32, 0, s>>>(S->partial + RED_BLOCKS, RED_BLOCKS, S->sc, SC_RZOLD);
      cudaMemcpyAsync(S->host_sc, S->sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s);
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve");
      ++it;
      if (std::sqrt(std::max(S->host_sc[SC_RR], 0.0)) <= tol_in || it >= o->max_iter) break;
      e = vcycle32_graph(M, S, z32, s);
      if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve: preconditioner");
      reduce32_to(r32, z32, n, S->partial, S->sc, SC_RZNEW, s);
      note_launch();
      pcg32_direction_kernel<<<G, 256, 0, s>>>(S->d32, z32, n, S->sc, 0);
      note_launch();
      copy_scalar_kernel<<<1, 1, 0, s>>>(S->sc, SC_RZ, SC_RZNEW);
    }
    // p += ||r|| e; r = b - A p in FP64
    note_launch();
    accumulate64_kernel<<<G, 256, 0, s>>>(p, S->e32, n, S->sc, SC_RN);
    e = launch_laplace<double>(M->v64, p, S->q, s);
    if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve: operator");
    cudaMemcpyAsync(S->r, S->b, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    note_launch();
    axpby_kernel<<<G, 256, 0, s>>>(S->r, S->q, -1.0, 1.0, n);
  }
  *iterations = it;
  return DGW_OK;
}

dgw_status pressure_solve(dgw_mesh *M, const double *b_in, double *p, const dgw_solve_opts *o, dgw_solve_info *info,
                          cudaStream_t cs) {
  dgw_solver *S = get_solver(M);
  if (!S) return set_error(DGW_ENOMEM, "dgw_pressure_solve: workspace allocation failed");
  cudaStream_t s = S->stream;
  cudaEventRecord(S->ev_in, cs);
  cudaStreamWaitEvent(s, S->ev_in, 0);
  const long n = M->np;
  const int G = grid_for(n);
  cudaError_t e;
  const unsigned long long dof0 = dof_counter();
  cudaEventRecord(S->ev0, s);
  // b <- b - mean(b); ||b||
  project_mean(b_in, S->b, n, S->partial, S->sc, SC_TMP, s);
  reduce_to(S->b, S->b, n, S->partial, S->sc, SC_BB, s);
  cudaMemsetAsync(p, 0, n * sizeof(double), s);
  cudaMemcpyAsync(S->r, S->b, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(S->host_sc, S->sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve");
  const double bnorm = std::sqrt(S->host_sc[SC_BB]);
  int it = 0;
  double rel = 0.0;
  dgw_status st = DGW_OK;
  if (bnorm == 0.0) {
    info->iterations = 0;
    info->rel_residual = 0.0;
    info->ms = 0.0f;
    info->dof_applies = 0.0;
    return DGW_OK;
  }
  if (o->mode == 1) {
    e = mg_setup(M, S, 1, o->cheb_degree > 0 ? o->cheb_degree : 5, s);
    if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve: multigrid setup");
    st = pressure_solve_mixed(M, S, o, p, bnorm, &it, s);
    if (st != DGW_OK && st != DGW_ENOTCONV) return st;
  }
  auto precondition = [&](const double *r, double *z) -> cudaError_t {
    if (o->mode == 2 || !S->mg_ready) {
      note_launch();
      jacobi_kernel<<<G, 256, 0, s>>>(r, M->diag64, z, n);
    } else {
      // the CG always preconditions S->r into S->z: the captured V-cycle reads and writes exactly those
      cudaError_t ee = (r == S->r && z == S->z) ? vcycle_graph(M, S, o->mode, s) : mg_vcycle(M, S, o->mode, r, z, s);
      if (ee != cudaSuccess) return ee;
    }
    return project_mean(z, z, n, S->partial, S->sc, SC_TMP, s);
  };
  if (o->mode == 0) {
    e = mg_setup(M, S, o->mode, o->cheb_degree > 0 ? o->cheb_degree : 5, s);
    if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve: multigrid setup");
  }
  if (o->mode != 1) {
    note_launch();
    copy_scalar_kernel<<<1, 1, 0, s>>>(S->sc, SC_RR, SC_BB);   // r = b: the preconditioner scales by rms(r)
    e = precondition(S->r, S->z);
    if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve: preconditioner");
    reduce_to(S->r, S->z, n, S->partial, S->sc, SC_RZNEW, s);
    note_launch();
    cg_direction_kernel<<<G, 256, 0, s>>>(S->d, S->z, n, S->sc, 1);
    note_launch();
    copy_scalar_kernel<<<1, 1, 0, s>>>(S->sc, SC_RZ, SC_RZNEW);
    for (it = 1; it <= o->max_iter; ++it) {
      e = launch_laplace<double>(M->v64, S->d, S->q, s);
      if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve: operator");
      reduce_to(S->d, S->q, n, S->partial, S->sc, SC_DQ, s);
      note_launch();
      cg_update_kernel<<<G, 256, 0, s>>>(p, S->r, S->d, S->q, n, S->sc);
      reduce_to(S->r, S->r, n, S->partial, S->sc, SC_RR, s);
      cudaMemcpyAsync(S->host_sc, S->sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s);
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve");
      rel = std::sqrt(std::max(S->host_sc[SC_RR], 0.0)) / bnorm;
      if (rel <= o->rtol) break;
      cudaMemcpyAsync(S->zold, S->z, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
      e = precondition(S->r, S->z);
      if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve: preconditioner");
      reduce_to(S->r, S->z, n, S->partial, S->sc, SC_RZNEW, s);
      reduce_to(S->r, S->zold, n, S->partial, S->sc, SC_RZOLD, s);
      note_launch();
      cg_direction_kernel<<<G, 256, 0, s>>>(S->d, S->z, n, S->sc, 0);
      note_launch();
      copy_scalar_kernel<<<1, 1, 0, s>>>(S->sc, SC_RZ, SC_RZNEW);
    }
    if (it > o->max_iter) { it = o->max_iter; st = DGW_ENOTCONV; }
  }
  // p <- p - mean(p); true residual in FP64
  project_mean(p, p, n, S->partial, S->sc, SC_TMP, s);
  launch_laplace<double>(M->v64, p, S->q, s);
  cudaMemcpyAsync(S->r, S->b, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  note_launch();
  axpby_kernel<<<G, 256, 0, s>>>(S->r, S->q, -1.0, 1.0, n);
  reduce_to(S->r, S->r, n, S->partial, S->sc, SC_RR, s);
  cudaEventRecord(S->ev1, s);
  cudaMemcpyAsync(S->host_sc, S->sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve");
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, S->ev0, S->ev1);
  cudaEventRecord(S->ev_out, s);
  cudaStreamWaitEvent(cs, S->ev_out, 0);
  info->iterations = it;
  info->rel_residual = std::sqrt(std::max(S->host_sc[SC_RR], 0.0)) / bnorm;
  info->ms = ms;
  info->dof_applies = (double)(dof_counter() - dof0);
  if (st == DGW_ENOTCONV) return set_error(DGW_ENOTCONV, "dgw_pressure_solve: max_iter reached");
  return DGW_OK;
}

}  // namespace dgw

void dgw_solver_free(dgw_mesh *M) {
  dgw_solver *S = M ? M->solver : nullptr;
  if (!S) return;
  dgw::mg_free(S);
  cudaFree(S->b); cudaFree(S->r); cudaFree(S->z); cudaFree(S->d); cudaFree(S->q); cudaFree(S->zold);
  cudaFree(S->partial); cudaFree(S->sc);
  cudaFree(S->d32); cudaFree(S->q32); cudaFree(S->e32);
  if (S->vgraph32) cudaGraphExecDestroy(S->vgraph32);
  if (S->host_sc) cudaFreeHost(S->host_sc);
  if (S->ev0) cudaEventDestroy(S->ev0);
  if (S->ev1) cudaEventDestroy(S->ev1);
  if (S->ev_in) cudaEventDestroy(S->ev_in);
  if (S->ev_out) cudaEventDestroy(S->ev_out);
  if (S->vgraph) cudaGraphExecDestroy(S->vgraph);
  if (S->stream) cudaStreamDestroy(S->stream);
  delete S;
  M->solver = nullptr;
}

extern "C" dgw_status dgw_pressure_solve(dgw_mesh_t M, const double *b, double *p, const dgw_solve_opts *opts,
                                         dgw_solve_info *info, void *stream) {
  if (!M || !b || !p || !opts || !info) return dgw::set_error(DGW_EINVAL, "dgw_pressure_solve: null argument");
  if (!(opts->rtol > 0) || opts->max_iter < 1 || opts->mode < 0 || opts->mode > 2)
    return dgw::set_error(DGW_EINVAL, "dgw_pressure_solve: rtol > 0, max_iter >= 1, mode in 0..2 required");
  if (opts->mode == 1 && !M->has32)
    return dgw::set_error(DGW_EINVAL, "dgw_pressure_solve: mixed mode needs a mesh with FP32 tables");
  return dgw::pressure_solve(M, b, p, opts, info, (cudaStream_t)stream);
}

extern "C" dgw_status dgw_solver_describe(dgw_mesh_t M, int mode, int *n_levels, double *lmax, int *cells,
                                          int max_levels, void *stream) {
  if (!M || !n_levels) return dgw::set_error(DGW_EINVAL, "dgw_solver_describe: null argument");
  if (mode < 0 || mode > 1) return dgw::set_error(DGW_EINVAL, "dgw_solver_describe: mode must be 0 or 1");
  if (mode == 1 && !M->has32) return dgw::set_error(DGW_EINVAL, "dgw_solver_describe: mesh has no FP32 tables");
  dgw_solver *S = dgw::get_solver(M);
  if (!S) return dgw::set_error(DGW_ENOMEM, "dgw_solver_describe: workspace allocation failed");
  cudaError_t e = dgw::mg_setup(M, S, mode, S->mg_cheb > 0 ? S->mg_cheb : 5, S->stream);
  if (e != cudaSuccess) return dgw::cuda_check(e, "dgw_solver_describe");
  (void)stream;
  *n_levels = dgw::mg_describe(S, lmax, cells, max_levels);
  return DGW_OK;
}
