// Pressure solve for callers that must not allocate device memory.
//
// dgw_pressure_solve keeps a per-mesh workspace that it allocates on first use. Some callers
// cannot let a library call cudaMalloc at solve time: code whose device memory is owned by a
// framework's caching allocator or by a fixed budget planned at start-up (a library allocation
// outside that pool can fail or push the pool out of memory), and latency-sensitive loops where
// cudaMalloc/cudaFree would implicitly synchronise the device and stall other streams. For them
// this file offers a Jacobi-preconditioned CG solve whose scratch vectors live in one file-scope
// device array of fixed size; the entry point itself allocates nothing. It reads one residual
// norm back to the host per iteration, so it synchronises the caller's stream every iteration.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <string>

#include "solver.h"

namespace dgw {

namespace {

constexpr long kNoAllocMaxNp = 131072;   // largest pressure vector (n_p) the scratch holds
constexpr int kNoAllocRed = 304;         // partial sums of the two-stage reductions
constexpr int kNoAllocMaxDevices = 64;
static_assert(kNoAllocRed >= RED_BLOCKS, "reduce_to writes RED_BLOCKS partial sums into the partial area");

// b (projected rhs), r, z, d, q vectors, reduction partials and the scalar slots.
constexpr size_t kScratchDoubles = 5 * (size_t)kNoAllocMaxNp + kNoAllocRed + SC_COUNT;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mutex;
double *g_scratch_addr[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array for the current device (looked up once per device; the
// host-side name of the array is only a stand-in and must never be passed to a kernel). The cached
// address belongs to the device's current context: a cudaDeviceReset between calls invalidates it.
cudaError_t scratch_address(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

__global__ void na_jacobi(const double *__restrict__ r, const double *__restrict__ dg, double *__restrict__ z, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) z[i] = r[i] / dg[i];
}

// p += alpha d, r -= alpha q, alpha = rz / dq
__global__ void na_update(double *__restrict__ p, double *__restrict__ r, const double *__restrict__ d,
                          const double *__restrict__ q, long n, const double *sc) {
  const double alpha = sc[SC_RZ] / sc[SC_DQ];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    p[i] += alpha * d[i];
    r[i] -= alpha * q[i];
  }
}

// d = z (first) or z + (rz_new / rz) d; then rz <- rz_new
__global__ void na_direction(double *__restrict__ d, const double *__restrict__ z, long n, const double *sc, int first) {
  const double beta = first ? 0.0 : sc[SC_RZNEW] / sc[SC_RZ];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    d[i] = first ? z[i] : z[i] + beta * d[i];
}

__global__ void na_shift(double *sc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) sc[SC_RZ] = sc[SC_RZNEW];
}

__global__ void na_sub(double *__restrict__ r, const double *__restrict__ b, const double *__restrict__ q, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) r[i] = b[i] - q[i];
}

inline int na_grid(long n) {
  long g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

// Reads one scalar slot back (synchronising s). A launch error left by the work queued before it
// is reported here, so each iteration's launches are checked once per read.
double read_scalar(const double *sc, int slot, cudaStream_t s, cudaError_t &e) {
  double v = 0.0;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, sc + slot, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return v;
}

}  // namespace

}  // namespace dgw

extern "C" dgw_status dgw_pressure_solve_jacobi_noalloc(dgw_mesh_t M, const double *b_in, double *p, double rtol,
                                                        int max_iter, dgw_solve_info *info, void *stream) {
  using namespace dgw;
  if (!M || !b_in || !p || !info) return set_error(DGW_EINVAL, "dgw_pressure_solve_jacobi_noalloc: null argument");
  if (!(rtol > 0) || max_iter < 1)
    return set_error(DGW_EINVAL, "dgw_pressure_solve_jacobi_noalloc: rtol > 0 and max_iter >= 1 required");
  const long n = M->np;
  if (n > kNoAllocMaxNp)
    return set_error(DGW_EINVAL, "dgw_pressure_solve_jacobi_noalloc: n_p = " + std::to_string(n) +
                                     " exceeds the fixed scratch limit of " + std::to_string(kNoAllocMaxNp) +
                                     " pressure DoFs; use dgw_pressure_solve");
  cudaStream_t s = (cudaStream_t)stream;
  {
    // every iteration reads the residual back and synchronises s, which a stream capture forbids:
    // refuse a capturing stream (or a capture elsewhere that makes s unusable) before any work
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(s, &cs);
    if (ce != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
      if (ce != cudaSuccess) (void)cudaGetLastError();
      return set_error(DGW_EINVAL, "dgw_pressure_solve_jacobi_noalloc: the stream is being captured; this solve "
                                   "synchronises its stream every iteration and cannot be captured");
    }
  }
  double *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve_jacobi_noalloc: scratch address");
  double *b = base, *r = b + kNoAllocMaxNp, *z = r + kNoAllocMaxNp, *d = z + kNoAllocMaxNp, *q = d + kNoAllocMaxNp;
  double *partial = q + kNoAllocMaxNp, *sc = partial + kNoAllocRed;
  const int G = na_grid(n);
  const auto t0 = std::chrono::steady_clock::now();
  const unsigned long long dof0 = dof_counter();
  // the array keeps the previous call's contents: clear the scalar slots and the output
  e = cudaMemsetAsync(sc, 0, SC_COUNT * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, n * sizeof(double), s);
  if (e == cudaSuccess) e = project_mean(b_in, b, n, partial, sc, SC_TMP, s);
  if (e == cudaSuccess) e = reduce_to(b, b, n, partial, sc, SC_BB, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  const double bnorm = std::sqrt(std::max(read_scalar(sc, SC_BB, s, e), 0.0));
  if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve_jacobi_noalloc");
  info->dof_applies = 0.0;
  if (bnorm == 0.0) {
    info->iterations = 0;
    info->rel_residual = 0.0;
    info->ms = 0.0f;
    return DGW_OK;
  }
  // z = D^-1 r projected to zero mean, rz_new = r.z; then the new search direction d
  auto precondition_and_direction = [&](int first) -> cudaError_t {
    note_launch();
    na_jacobi<<<G, 256, 0, s>>>(r, M->diag64, z, n);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) err = project_mean(z, z, n, partial, sc, SC_TMP, s);
    if (err == cudaSuccess) err = reduce_to(r, z, n, partial, sc, SC_RZNEW, s);
    if (err != cudaSuccess) return err;
    note_launches(2);
    na_direction<<<G, 256, 0, s>>>(d, z, n, sc, first);
    na_shift<<<1, 32, 0, s>>>(sc);
    return cudaGetLastError();
  };
  e = precondition_and_direction(1);
  if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve_jacobi_noalloc: preconditioner");
  int it = 0;
  dgw_status st = DGW_OK;
  for (it = 1; it <= max_iter; ++it) {
    e = launch_laplace<double>(M->v64, d, q, s);
    if (e == cudaSuccess) e = reduce_to(d, q, n, partial, sc, SC_DQ, s);
    if (e == cudaSuccess) {
      note_launch();
      na_update<<<G, 256, 0, s>>>(p, r, d, q, n, sc);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = reduce_to(r, r, n, partial, sc, SC_RR, s);
    const double rel = std::sqrt(std::max(read_scalar(sc, SC_RR, s, e), 0.0)) / bnorm;
    if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve_jacobi_noalloc: iteration");
    if (rel <= rtol) break;
    e = precondition_and_direction(0);
    if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve_jacobi_noalloc: preconditioner");
  }
  if (it > max_iter) { it = max_iter; st = DGW_ENOTCONV; }
  // zero-mean solution and its true FP64 residual
  e = project_mean(p, p, n, partial, sc, SC_TMP, s);
  if (e == cudaSuccess) e = launch_laplace<double>(M->v64, p, q, s);
  if (e == cudaSuccess) {
    note_launch();
    na_sub<<<G, 256, 0, s>>>(r, b, q, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = reduce_to(r, r, n, partial, sc, SC_RR, s);
  const double rr = read_scalar(sc, SC_RR, s, e);
  if (e != cudaSuccess) return cuda_check(e, "dgw_pressure_solve_jacobi_noalloc");
  info->iterations = it;
  info->rel_residual = std::sqrt(std::max(rr, 0.0)) / bnorm;
  info->ms = (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  info->dof_applies = (double)(dof_counter() - dof0);
  if (st == DGW_ENOTCONV) return set_error(DGW_ENOTCONV, "dgw_pressure_solve_jacobi_noalloc: max_iter reached");
  return DGW_OK;
}
