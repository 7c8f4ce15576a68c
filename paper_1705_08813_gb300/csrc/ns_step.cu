// One time step of the dual-splitting scheme (Sec. 4.1 with the Galerkin forms of Sec. 4.2):
//   0. (optional) wall model: tau_w,B from u^n, the velocity history L2-projected onto the new space
//      and the convective history recomputed in it (Sec. 3.2)
//   1. explicit convective step (eq. convstepspat), BDF/extrapolation of order J = 2 (J = 1 in the
//      first step), with the exact cell-wise inverse mass:
//        u^ = (sum_i alpha_i u^{n-i} + dt f - dt M^-1 sum_i beta_i F^c(u^{n-i})) / gamma_0
//   2. pressure Poisson equation (eq. poissonspat): A p = (gamma_0 / dt) (-C u^) + (q, g)_walls with the
//      high-order Neumann data g of eq. bc_d_pres (vorticities omega^{n-i} = M^-1 (v, curl u^{n-i})),
//      or g = 0
//   3. projection (eq. projectionspat): (M + D) u^^ = M u^ - (dt / gamma_0) P(v, p), D with tau_D from
//      u^n, solved by CG preconditioned with the exact inverse mass
//   4. viscous step (eq. helmholtzspat): (gamma_0 / dt) M u^{n+1} - F^nu(u^{n+1}) = (gamma_0 / dt) M u^^,
//      nu_t frozen from u^n, restarted GMRES
// Constant time step, or (adaptive_dt) the CFL step dt_n = min(dt, Cr / (k^1.5 rate(u^n))) with the
// BDF2 / extrapolation constants of the step ratio. Every operator is a library kernel; the host
// sequences them.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "dgw_internal.h"

void dgw_helm_free(dgw_mesh *M);

struct dgw_ns {
  dgw_mesh *M = nullptr;
  dgw_ns_params P{};
  long nu = 0, np = 0;
  int steps = 0;
  double dt_prev = 0.0;                 // the previous step size (variable-step constants)
  double *u[2] = {nullptr, nullptr};    // u^n, u^{n-1}
  double *fc[2] = {nullptr, nullptr};   // F^c(u^n), F^c(u^{n-1})
  double *om[2] = {nullptr, nullptr};   // vorticities of u^n, u^{n-1} (high-order pressure data)
  double *p = nullptr, *b = nullptr;
  double *uh = nullptr, *uhh = nullptr, *w = nullptr, *x = nullptr, *t1 = nullptr, *t2 = nullptr;
  double *f = nullptr;                  // body force as a velocity field (standard coefficients)
  double *tau_d = nullptr, *tau_nodes = nullptr;
  double *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_q = nullptr;
  double *partial = nullptr;
  double *cg_sc = nullptr, *cg_host = nullptr;   // projection CG scalars on the device and their host copy
  std::vector<void *> allocs;
};

namespace dgw {
namespace {

constexpr int kDotBlocks = 512;

// out = a x + b y (+ c z)
__global__ void lincomb_kernel(double *__restrict__ out, double a, const double *__restrict__ x, double b,
                               const double *__restrict__ y, double c, const double *__restrict__ z, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double v = a * x[i];
    if (y) v += b * y[i];
    if (z) v += c * z[i];
    out[i] = v;
  }
}

// partial[blk] = sum of x[i] y[i] over a fixed stride pattern (deterministic)
__global__ void dot_partial_kernel(const double *__restrict__ x, const double *__restrict__ y, long n,
                                   double *__restrict__ partial) {
  __shared__ double red[256];
  double s = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) s += x[i] * y[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Projection CG with the scalars on the device: slots of cg_sc
enum { CG_RR = 0, CG_PQ, CG_RZ, CG_RZNEW, CG_DONE, CG_ITER, CG_TARGET, CG_COUNT };

// sc[slot] = sum of the partials; with flag: the convergence test sqrt(rr) <= target raises CG_DONE
__global__ void cg_finish_kernel(const double *__restrict__ partial, int nb, double *__restrict__ sc, int slot, int flag) {
  __shared__ double red[512];
  red[threadIdx.x] = threadIdx.x < nb ? partial[threadIdx.x] : 0.0;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sc[slot] = red[0];
    if (flag && sc[CG_DONE] == 0.0 && sqrt(red[0]) <= sc[CG_TARGET]) sc[CG_DONE] = 1.0;
  }
}

// x += alpha p, r -= alpha q with alpha = rz / pq (nothing once the iteration has converged)
__global__ void cg_update_kernel(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                                 const double *__restrict__ q, long n, double *__restrict__ sc) {
  if (sc[CG_DONE] != 0.0) return;
  const double alpha = sc[CG_RZ] / sc[CG_PQ];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    r[i] -= alpha * q[i];
  }
}

// p = z + (rz_new / rz) p
__global__ void cg_direction_kernel(double *__restrict__ p, const double *__restrict__ z, long n,
                                    const double *__restrict__ sc) {
  if (sc[CG_DONE] != 0.0) return;
  const double beta = sc[CG_RZNEW] / sc[CG_RZ];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// rz <- rz_new and the iteration count, after every block of the direction update has read rz
__global__ void cg_shift_kernel(double *sc) {
  if (sc[CG_DONE] != 0.0) return;
  sc[CG_RZ] = sc[CG_RZNEW];
  sc[CG_ITER] += 1.0;
}

// force field: every standard coefficient of component a equals f[a]; enrichment zero
__global__ void force_field_kernel(double *__restrict__ f, long np, int n3, double f0, double f1, double f2, long nu) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nu; i += (long)gridDim.x * blockDim.x) {
    if (i >= 3 * np) { f[i] = 0.0; continue; }
    const int a = (int)((i / n3) % 3);
    f[i] = a == 0 ? f0 : (a == 1 ? f1 : f2);
  }
}

int grid_of(long n) { return (int)std::min<long>(std::max<long>((n + 255) / 256, 1), 152 * 8); }

}  // namespace
}  // namespace dgw

using namespace dgw;

namespace {

dgw_status ns_fail(cudaError_t e, const char *what) { return cuda_check(e, what); }

cudaError_t lincomb(double *out, double a, const double *x, double b, const double *y, double c, const double *z, long n,
                    cudaStream_t s) {
  note_launch();
  lincomb_kernel<<<grid_of(n), 256, 0, s>>>(out, a, x, b, y, c, z, n);
  return cudaGetLastError();
}

// y = (M + D) x
dgw_status apply_md(dgw_ns *S, const double *x, double *y, cudaStream_t s) {
  dgw_status st = dgw_apply_mass(S->M, DGW_FP64, x, y, s);
  if (st == DGW_OK) st = dgw_apply_divdiv(S->M, S->tau_d, x, S->t2, s);
  if (st == DGW_OK) st = cuda_check(lincomb(y, 1.0, y, 1.0, S->t2, 0.0, nullptr, S->nu, s), "dgw_ns_step");
  return st;
}

// sc[slot] = x . y on the device (with flag: the convergence test of sc[CG_RR])
cudaError_t dot_dev(dgw_ns *S, const double *x, const double *y, long n, int slot, int flag, cudaStream_t s) {
  note_launches(2);
  dot_partial_kernel<<<kDotBlocks, 256, 0, s>>>(x, y, n, S->partial);
  cg_finish_kernel<<<1, 512, 0, s>>>(S->partial, kDotBlocks, S->cg_sc, slot, flag);
  return cudaGetLastError();
}

// (M + D) x = rhs by CG preconditioned with M^-1; x holds the initial guess. The scalars stay on the
// device: each iteration is launches only, a converged iteration leaves x, r and p unchanged, and the
// host reads the convergence flag and the iteration count every kCgCheck iterations (at most
// kCgCheck - 1 operator applies after convergence; the result and the count are those of a test in
// every iteration).
constexpr int kCgCheck = 4;
dgw_status projection_cg(dgw_ns *S, const double *rhs, double *x, cudaStream_t s, int *iters) {
  const long n = S->nu;
  const int G = grid_of(n);
  dgw_status st = apply_md(S, x, S->cg_q, s);
  cudaError_t e = cudaSuccess;
  if (st == DGW_OK) e = lincomb(S->cg_r, 1.0, rhs, -1.0, S->cg_q, 0.0, nullptr, n, s);
  if (st == DGW_OK && e == cudaSuccess) e = dot_dev(S, rhs, rhs, n, CG_RR, 0, s);
  if (st == DGW_OK && e == cudaSuccess) st = dgw_apply_inverse_mass(S->M, S->cg_r, S->cg_z, s);
  if (st == DGW_OK && e == cudaSuccess) e = cudaMemcpyAsync(S->cg_p, S->cg_z, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (st == DGW_OK && e == cudaSuccess) e = dot_dev(S, S->cg_r, S->cg_z, n, CG_RZ, 0, s);
  if (st == DGW_OK && e == cudaSuccess) e = cudaMemcpyAsync(S->cg_host, S->cg_sc, CG_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (st == DGW_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (st != DGW_OK) return st;
  if (e != cudaSuccess) return ns_fail(e, "dgw_ns_step");
  const double bb = S->cg_host[CG_RR];
  if (bb == 0.0) {   // x already solves the system exactly
    *iters = 0;
    return DGW_OK;
  }
  S->cg_host[CG_TARGET] = S->P.rtol_projection * std::sqrt(bb);
  S->cg_host[CG_DONE] = 0.0;
  S->cg_host[CG_ITER] = 0.0;
  e = cudaMemcpyAsync(S->cg_sc, S->cg_host, CG_COUNT * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return ns_fail(e, "dgw_ns_step");
  int launched = 0;
  for (;;) {
    for (int k = 0; k < kCgCheck && launched < S->P.max_iter + 1; ++k, ++launched) {
      e = dot_dev(S, S->cg_r, S->cg_r, n, CG_RR, 1, s);
      if (e != cudaSuccess) return ns_fail(e, "dgw_ns_step");
      st = apply_md(S, S->cg_p, S->cg_q, s);
      if (st != DGW_OK) return st;
      e = dot_dev(S, S->cg_p, S->cg_q, n, CG_PQ, 0, s);
      if (e == cudaSuccess) {
        note_launch();
        cg_update_kernel<<<G, 256, 0, s>>>(x, S->cg_r, S->cg_p, S->cg_q, n, S->cg_sc);
        e = cudaGetLastError();
      }
      if (e != cudaSuccess) return ns_fail(e, "dgw_ns_step");
      st = dgw_apply_inverse_mass(S->M, S->cg_r, S->cg_z, s);
      if (st != DGW_OK) return st;
      e = dot_dev(S, S->cg_r, S->cg_z, n, CG_RZNEW, 0, s);
      if (e == cudaSuccess) {
        note_launches(2);
        cg_direction_kernel<<<G, 256, 0, s>>>(S->cg_p, S->cg_z, n, S->cg_sc);
        cg_shift_kernel<<<1, 1, 0, s>>>(S->cg_sc);
        e = cudaGetLastError();
      }
      if (e != cudaSuccess) return ns_fail(e, "dgw_ns_step");
    }
    e = cudaMemcpyAsync(S->cg_host, S->cg_sc, CG_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ns_fail(e, "dgw_ns_step");
    if (S->cg_host[CG_DONE] != 0.0) break;
    if (launched > S->P.max_iter) break;
  }
  const int it = (int)S->cg_host[CG_ITER];
  *iters = it;
  if (S->cg_host[CG_DONE] == 0.0) return set_error(DGW_ENOTCONV, "dgw_ns_step: projection CG reached max_iter");
  return DGW_OK;
}

void ns_free(dgw_ns *S) {
  if (!S) return;
  for (void *p : S->allocs) cudaFree(p);
  if (S->cg_host) cudaFreeHost(S->cg_host);
  delete S;
}

}  // namespace

extern "C" {

dgw_status dgw_ns_create(dgw_mesh_t M, const dgw_ns_params *params, const double *u0, void *stream, dgw_ns_t *out) {
  if (!M || !params || !u0 || !out) return set_error(DGW_EINVAL, "dgw_ns_create: null argument");
  if (!(params->dt > 0.0) || !(params->cr > 0.0) || !(params->rtol_pressure > 0.0) ||
      !(params->rtol_projection > 0.0) || !(params->rtol_viscous > 0.0) || params->max_iter < 1)
    return set_error(DGW_EINVAL, "dgw_ns_create: dt, cr, tolerances and max_iter must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  dgw_ns *S = new dgw_ns();
  S->M = M;
  S->P = *params;
  S->nu = M->nu;
  S->np = M->np;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](double **p, size_t count) {
    void *q = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(double));
    if (e == cudaSuccess) {
      S->allocs.push_back(q);
      *p = (double *)q;
      e = cudaMemsetAsync(q, 0, std::max<size_t>(count, 1) * sizeof(double), s);
    }
  };
  for (int i = 0; i < 2; ++i) { alloc(&S->u[i], S->nu); alloc(&S->fc[i], S->nu); alloc(&S->om[i], S->nu); }
  for (double **p : {&S->uh, &S->uhh, &S->w, &S->x, &S->t1, &S->t2, &S->f, &S->cg_r, &S->cg_z, &S->cg_p, &S->cg_q})
    alloc(p, S->nu);
  alloc(&S->p, S->np);
  alloc(&S->b, S->np);
  alloc(&S->tau_d, M->nc);
  alloc(&S->tau_nodes, (size_t)2 * M->P.nx * M->P.nz);
  alloc(&S->partial, kDotBlocks + 1);
  alloc(&S->cg_sc, CG_COUNT);
  if (e == cudaSuccess) e = cudaMallocHost(&S->cg_host, CG_COUNT * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->u[0], u0, S->nu * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) {
    note_launch();
    force_field_kernel<<<grid_of(S->nu), 256, 0, s>>>(S->f, S->np, M->n1 * M->n1 * M->n1, params->force[0],
                                                      params->force[1], params->force[2], S->nu);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    ns_free(S);
    return cuda_check(e, "dgw_ns_create");
  }
  *out = S;
  return DGW_OK;
}

dgw_status dgw_ns_destroy(dgw_ns_t S) {
  ns_free(S);
  return DGW_OK;
}

dgw_status dgw_ns_state(dgw_ns_t S, const double **u, const double **p, int *steps) {
  if (!S) return set_error(DGW_EINVAL, "dgw_ns_state: null handle");
  if (u) *u = S->u[0];
  if (p) *p = S->p;
  if (steps) *steps = S->steps;
  return DGW_OK;
}

dgw_status dgw_ns_copy_state(dgw_ns_t S, double *u, double *p, void *stream) {
  if (!S) return set_error(DGW_EINVAL, "dgw_ns_copy_state: null handle");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (u) e = cudaMemcpyAsync(u, S->u[0], S->nu * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && p) e = cudaMemcpyAsync(p, S->p, S->np * sizeof(double), cudaMemcpyDeviceToDevice, s);
  return cuda_check(e, "dgw_ns_copy_state");
}

dgw_status dgw_ns_step(dgw_ns_t S, dgw_ns_step_info *info, void *stream) {
  if (!S) return set_error(DGW_EINVAL, "dgw_ns_step: null handle");
  cudaStream_t s = (cudaStream_t)stream;
  dgw_mesh *M = S->M;
  const auto t0 = std::chrono::steady_clock::now();
  const long nu = S->nu;
  const bool second = S->steps > 0;
  dgw_ns_step_info inf{};
  dgw_status st = DGW_OK;
  cudaError_t e = cudaSuccess;
  // step size: constant, or the CFL step of u^n (Sec. 4.1, Cr = cr)
  double dt = S->P.dt;
  if (S->P.adaptive_dt) {
    double rate = 0.0;
    st = dgw_cfl_rate(M, S->u[0], &rate, s);
    if (st != DGW_OK) return st;
    if (rate > 0.0) dt = std::min(dt, S->P.cr / (std::pow((double)M->P.degree, 1.5) * rate));
  }
  // BDF2 / extrapolation of order 2 (order 1 in the first step); step ratio w = dt_n / dt_{n-1}
  double g0 = 1.0, a0 = 1.0, a1 = 0.0, b0 = 1.0, b1 = 0.0;
  if (second) {
    const double w = S->P.adaptive_dt ? dt / S->dt_prev : 1.0;
    if (w == 1.0) {
      g0 = 1.5; a0 = 2.0; a1 = -0.5; b0 = 2.0; b1 = -1.0;
    } else {
      g0 = (1.0 + 2.0 * w) / (1.0 + w);
      a0 = 1.0 + w;
      a1 = -w * w / (1.0 + w);
      b0 = 1.0 + w;
      b1 = -w;
    }
  }
  // 0. wall model: new tau_w and the history moved into the new space
  if (S->P.update_wall_model && M->ne > 0) {
    st = dgw_wall_shear_stress(M, S->u[0], S->tau_nodes, s);
    if (st == DGW_OK) {
      // the wall law needs tau_w > 0 at every node
      std::vector<double> h((size_t)2 * M->P.nx * M->P.nz);
      e = cudaMemcpyAsync(h.data(), S->tau_nodes, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_check(e, "dgw_ns_step");
      for (double v : h)
        if (!(v > 0.0) || !std::isfinite(v))
          return set_error(DGW_EDEVICE, "dgw_ns_step: the wall shear stress vanished at a wall node");
    }
    if (st == DGW_OK) {
      int bad = -1;
      const double *olds[2] = {S->u[0], S->u[1]};
      double *news[2] = {S->u[0], S->u[1]};
      st = cuda_check(launch_projection(M, S->tau_nodes, second ? 2 : 1, olds, news, s, &bad), "dgw_ns_step");
      if (st == DGW_OK && bad >= 0) st = set_error(DGW_EDEVICE, "dgw_ns_step: singular wall-cell mass matrix");
      dgw_helm_free(M);
    }
    if (st == DGW_OK && second) st = dgw_apply_convective(M, DGW_FP64, S->u[1], S->fc[1], s);
    if (st == DGW_OK && second && S->P.pressure_bc) {   // vorticity of the projected u^{n-1}
      st = dgw_apply_curl(M, S->u[1], S->t1, s);
      if (st == DGW_OK) st = dgw_apply_inverse_mass(M, S->t1, S->om[1], s);
    }
    if (st != DGW_OK) return st;
  }
  if (S->P.pressure_bc) {   // vorticity of u^n
    st = dgw_apply_curl(M, S->u[0], S->t1, s);
    if (st == DGW_OK) st = dgw_apply_inverse_mass(M, S->t1, S->om[0], s);
    if (st != DGW_OK) return st;
  }
  // 1. convective step
  st = dgw_update_eddy_viscosity(M, S->u[0], s);
  if (st == DGW_OK) st = dgw_tau_divdiv(M, S->u[0], dt, S->P.cr, S->tau_d, s);
  if (st == DGW_OK) st = dgw_apply_convective(M, DGW_FP64, S->u[0], S->fc[0], s);
  if (st == DGW_OK) st = cuda_check(lincomb(S->w, b0, S->fc[0], b1, second ? S->fc[1] : nullptr, 0.0, nullptr, nu, s),
                                    "dgw_ns_step");
  if (st == DGW_OK) st = dgw_apply_inverse_mass(M, S->w, S->x, s);
  if (st == DGW_OK) st = cuda_check(lincomb(S->t1, a0 / g0, S->u[0], a1 / g0, second ? S->u[1] : nullptr, dt / g0, S->f,
                                            nu, s), "dgw_ns_step");
  if (st == DGW_OK) st = cuda_check(lincomb(S->uh, 1.0, S->t1, -dt / g0, S->x, 0.0, nullptr, nu, s), "dgw_ns_step");
  // 2. pressure
  if (st == DGW_OK) st = dgw_apply_divergence(M, S->uh, S->b, s);
  if (st == DGW_OK) st = cuda_check(lincomb(S->b, g0 / dt, S->b, 0.0, nullptr, 0.0, nullptr, S->np, s), "dgw_ns_step");
  if (st == DGW_OK && S->P.pressure_bc)
    st = dgw_add_pressure_neumann(M, S->u[0], S->om[0], b0, second ? S->u[1] : nullptr, second ? S->om[1] : nullptr,
                                  second ? b1 : 0.0, S->P.force, S->b, s);
  if (st == DGW_OK) {
    dgw_solve_opts o{};
    o.rtol = S->P.rtol_pressure;
    o.max_iter = S->P.max_iter;
    o.mode = S->P.pressure_mode;
    o.cheb_degree = 5;
    dgw_solve_info si{};
    st = dgw_pressure_solve(M, S->b, S->p, &o, &si, s);
    inf.pressure_iterations = si.iterations;
  }
  // 3. projection
  if (st == DGW_OK) st = dgw_apply_mass(M, DGW_FP64, S->uh, S->t1, s);
  if (st == DGW_OK) st = dgw_apply_gradient(M, S->p, S->t2, s);
  if (st == DGW_OK) st = cuda_check(lincomb(S->w, 1.0, S->t1, -dt / g0, S->t2, 0.0, nullptr, nu, s), "dgw_ns_step");
  if (st == DGW_OK) e = cudaMemcpyAsync(S->uhh, S->uh, nu * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (st == DGW_OK && e != cudaSuccess) st = cuda_check(e, "dgw_ns_step");
  if (st == DGW_OK) st = projection_cg(S, S->w, S->uhh, s, &inf.projection_iterations);
  // 4. viscous step: u^{n+1} goes into u[1], which then becomes u^n
  if (st == DGW_OK) st = dgw_apply_mass(M, DGW_FP64, S->uhh, S->w, s);
  if (st == DGW_OK) st = cuda_check(lincomb(S->w, g0 / dt, S->w, 0.0, nullptr, 0.0, nullptr, nu, s), "dgw_ns_step");
  if (st == DGW_OK) e = cudaMemcpyAsync(S->x, S->uhh, nu * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (st == DGW_OK && e != cudaSuccess) st = cuda_check(e, "dgw_ns_step");
  if (st == DGW_OK) {
    dgw_helmholtz_opts ho{};
    ho.rtol = S->P.rtol_viscous;
    ho.max_iter = S->P.max_iter;
    ho.restart = 30;
    dgw_solve_info hi{};
    st = dgw_helmholtz_solve(M, g0 / dt, S->w, S->x, &ho, &hi, s);
    inf.viscous_iterations = hi.iterations;
  }
  if (st != DGW_OK) return st;
  // history: u^{n-1} <- u^n, u^n <- u^{n+1}; F^c(u^{n-1}) <- F^c(u^n)
  std::swap(S->u[0], S->u[1]);
  e = cudaMemcpyAsync(S->u[0], S->x, nu * sizeof(double), cudaMemcpyDeviceToDevice, s);
  std::swap(S->fc[0], S->fc[1]);
  std::swap(S->om[0], S->om[1]);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(e, "dgw_ns_step");
  S->steps++;
  S->dt_prev = dt;
  inf.dt = dt;
  inf.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  return DGW_OK;
}

}  // extern "C"
