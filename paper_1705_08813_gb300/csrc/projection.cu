// Cell-wise L2 projection of the velocity onto the enrichment space of a new nodal wall shear stress
// (Sec. 3.2, eq. l2): in every enriched cell, find u_new in V_new with (v, u_new) = (v, u_old) for all
// v in V_new, per component, integrated with the cell's velocity point set (k+1 Gauss points
// in-plane, q_w wall-normal). The other cells keep their space, so their coefficients are copied.
//
// Three steps on the stream:
//   1. project_eval_kernel (old wall tables): u_old at every point of every enriched cell.
//   2. new nodal tau_w: the wall tables are rebuilt (the enrichment space changes).
//   3. project_solve_kernel (new wall tables), one CTA per enriched cell: the cell's mass matrix of
//      V_new (N = (k+1)^3 + nef unknowns per component, the same matrix for the three components)
//      is assembled with the standard-standard block by sum factorisation over the three point
//      axes, the right-hand sides from the stored point values, then factorised by Cholesky in a
//      global scratch block and solved for the three components.
// The cell systems are ill-conditioned where a wall cell spans few wall units (psi N_B close to the
// polynomials); a non-positive pivot sets the error word and the cell is left unsolved. A cell
// whose wall model is switched off in the new space solves its standard block only (enrichment
// coefficients zero); every wall cell integrates with the enriched point set either way.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "dgw_internal.h"
#include "metric.cuh"
#include "sumfac.cuh"

namespace dgw {
namespace {

// u_old at the points (x fastest, wall-normal set in y) of enriched cell e: P[e][t][3]
__global__ void project_eval_kernel(MeshView<double> m, const int *__restrict__ enr_cell, const double *__restrict__ u,
                                    const double *__restrict__ wt_vol, int nvol, double *__restrict__ P) {
  const Basis<double> &B = *m.basis;
  const int n = m.n1, n3 = n * n * n, e = blockIdx.x, cell = enr_cell[e];
  __shared__ double su[3 * NMAX * NMAX * NMAX], ce[24];
  for (int t = threadIdx.x; t < 3 * n3; t += blockDim.x) su[t] = u[(size_t)cell * 3 * n3 + t];
  const bool on = m.enr[cell] >= 0;   // switched off: the old space has no enrichment here
  for (int t = threadIdx.x; t < 24; t += blockDim.x)
    ce[t] = on ? u[3 * m.np + (size_t)e * 3 * m.nef + (m.nef == 8 ? t : t >> 3)] : 0.0;
  __syncthreads();
  const int sx = m.full_q ? QSET_WALL : QSET_LIN;   // in-plane set of the wall cells
  const int q0 = B.q[sx], q1 = B.q[QSET_WALL];
  const double *S0 = B.S[sx], *Sw = B.S[QSET_WALL];
  for (int t = threadIdx.x; t < nvol; t += blockDim.x) {
    const int i0 = t % q0, i1 = (t / q0) % q1, i2 = t / (q0 * q1);
    const double xi[3] = {B.x[sx][i0], B.x[QSET_WALL][i1], B.x[sx][i2]};
    double val[3] = {0.0, 0.0, 0.0};
    for (int cc = 0; cc < n; ++cc)
      for (int bb = 0; bb < n; ++bb) {
        const double s12 = Sw[i1 * n + bb] * S0[i2 * n + cc];
        for (int aa = 0; aa < n; ++aa) {
          const double ph = S0[i0 * n + aa] * s12;
          const int node = aa + n * (bb + n * cc);
          for (int a = 0; a < 3; ++a) val[a] += ph * su[a * n3 + node];
        }
      }
    const double psi = wt_vol[((size_t)e * nvol + t) * WT];
    double N[8], dN[8][3];
    q1_weights(xi, N, dN);
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int v = 0; v < 8; ++v) s += ce[a * 8 + v] * N[v];
      P[((size_t)e * nvol + t) * 3 + a] = val[a] + psi * s;
    }
  }
}

struct ProjLayout {
  int W, PSI, T1, T2, RHS, COL, total;
};

__host__ __device__ inline ProjLayout proj_layout(int n, int q0, int q1, int nef) {
  ProjLayout L;
  const int npts = q0 * q1 * q0, N = n * n * n + nef;
  int o = 0;
  L.W = o; o += npts;
  L.PSI = o; o += npts;
  L.T1 = o; o += q0 * q1 * n * n;
  L.T2 = o; o += q0 * n * n * n * n;
  L.RHS = o; o += 3 * N;
  L.COL = o; o += N;
  L.total = o;
  return L;
}

__device__ __forceinline__ double enr_weight(int nef, int v, const double xi[3]) {
  if (nef == 1) return 1.0;
  return ((v & 1) ? xi[0] : 1.0 - xi[0]) * ((v & 2) ? xi[1] : 1.0 - xi[1]) * ((v & 4) ? xi[2] : 1.0 - xi[2]);
}

__global__ void project_solve_kernel(MeshView<double> m, const int *__restrict__ enr_cell,
                                     const double *__restrict__ wt_vol, int nvol, const double *__restrict__ P,
                                     double *__restrict__ Ag, double *__restrict__ u_new, int *__restrict__ err) {
  extern __shared__ double sm[];
  const Basis<double> &B = *m.basis;
  const int n = m.n1, n2 = n * n, n3 = n2 * n, N = n3 + m.nef;
  const int sx = m.full_q ? QSET_WALL : QSET_LIN;   // in-plane set of the wall cells
  const int q0 = B.q[sx], q1 = B.q[QSET_WALL], npts = q0 * q1 * q0;
  const ProjLayout L = proj_layout(n, q0, q1, m.nef);
  double *W = sm + L.W, *PSI = sm + L.PSI, *T1 = sm + L.T1, *T2 = sm + L.T2, *R = sm + L.RHS, *col = sm + L.COL;
  const int e = blockIdx.x, c = enr_cell[e], tid = threadIdx.x, nt = blockDim.x;
  // P == nullptr: factorise only (the inverse mass of cells with the wall model switched on)
  const bool rhs = P != nullptr;
  if (!rhs && m.enr[c] < 0) return;
  // switched off in the new space: the standard block alone (stride N kept), zero enrichment
  const int nef = m.enr[c] >= 0 ? m.nef : 0, Nc = n3 + nef;
  double *A = Ag + (size_t)e * N * N;
  const double *S0 = B.S[sx], *Sw = B.S[QSET_WALL];
  const double *w0 = B.w[sx], *w1 = B.w[QSET_WALL];
  // 0. weights |det J| w at the points and psi_new
  const double hbox = m.geo == GEO_CURVED ? 0.0 : m.hx * m.hy[(c / m.nx) % m.ny] * m.hz;
  const int colm = m.geo == GEO_CURVED ? metric_col(m, c) : 0;
  for (int t = tid; t < npts; t += nt) {
    const int i0 = t % q0, i1 = (t / q0) % q1, i2 = t / (q0 * q1);
    const double det = m.geo == GEO_CURVED ? fabs(vol_rec(m, B, colm, sx, QSET_WALL, i0, i1)[9]) : hbox;
    W[t] = det * w0[i0] * w1[i1] * w0[i2];
    PSI[t] = wt_vol[((size_t)e * nvol + t) * WT];
  }
  __syncthreads();
  // 1. T1[t0][t1][c][c'] = sum_t2 W S0[t2][c] S0[t2][c']
  for (int p = tid; p < q0 * q1 * n2; p += nt) {
    const int cc = p % n2, t01 = p / n2, t0 = t01 % q0, t1 = t01 / q0;
    const int c1 = cc / n, c2 = cc % n;
    double s = 0.0;
    for (int t2 = 0; t2 < q0; ++t2) s += W[t0 + q0 * (t1 + q1 * t2)] * S0[t2 * n + c1] * S0[t2 * n + c2];
    T1[(t0 * q1 + t1) * n2 + cc] = s;
  }
  __syncthreads();
  // 2. T2[t0][b][b'][c][c'] = sum_t1 T1[t0][t1][c][c'] Sw[t1][b] Sw[t1][b']
  for (int p = tid; p < q0 * n2 * n2; p += nt) {
    const int cc = p % n2, bb = (p / n2) % n2, t0 = p / (n2 * n2);
    const int b1 = bb / n, b2 = bb % n;
    double s = 0.0;
    for (int t1 = 0; t1 < q1; ++t1) s += T1[(t0 * q1 + t1) * n2 + cc] * Sw[t1 * n + b1] * Sw[t1 * n + b2];
    T2[p] = s;
  }
  __syncthreads();
  // 3. standard block: A[(a,b,c)][(a',b',c')] = sum_t0 T2[t0][b b'][c c'] S0[t0][a] S0[t0][a']
  for (int p = tid; p < n3 * n3; p += nt) {
    const int i = p / n3, j = p % n3;
    const int a1 = i % n, b1 = (i / n) % n, c1 = i / n2;
    const int a2 = j % n, b2 = (j / n) % n, c2 = j / n2;
    const int off = (b1 * n + b2) * n2 + c1 * n + c2;
    double s = 0.0;
    for (int t0 = 0; t0 < q0; ++t0) s += T2[t0 * n2 * n2 + off] * S0[t0 * n + a1] * S0[t0 * n + a2];
    A[(size_t)i * N + j] = s;
  }
  // 4. enriched-standard blocks and the standard right-hand sides
  for (int p = tid; p < n3 * (nef + (rhs ? 3 : 0)); p += nt) {
    const int i = p % n3, k = p / n3;   // k < nef: enriched column v = k; else component k - nef
    const int a1 = i % n, b1 = (i / n) % n, c1 = i / n2;
    double s = 0.0;
    for (int t = 0; t < npts; ++t) {
      const int i0 = t % q0, i1 = (t / q0) % q1, i2 = t / (q0 * q1);
      const double ph = S0[i0 * n + a1] * Sw[i1 * n + b1] * S0[i2 * n + c1] * W[t];
      if (k < nef) {
        const double xi[3] = {B.x[sx][i0], B.x[QSET_WALL][i1], B.x[sx][i2]};
        s += ph * PSI[t] * enr_weight(nef, k, xi);
      } else {
        s += ph * P[((size_t)e * npts + t) * 3 + (k - nef)];
      }
    }
    if (k < nef) {
      A[(size_t)i * N + n3 + k] = s;
      A[(size_t)(n3 + k) * N + i] = s;
    } else {
      R[(k - nef) * N + i] = s;
    }
  }
  // 5. enriched-enriched block and the enriched right-hand sides
  for (int p = tid; p < nef * (nef + (rhs ? 3 : 0)); p += nt) {
    const int v = p % nef, k = p / nef;
    double s = 0.0;
    for (int t = 0; t < npts; ++t) {
      const int i0 = t % q0, i1 = (t / q0) % q1, i2 = t / (q0 * q1);
      const double xi[3] = {B.x[sx][i0], B.x[QSET_WALL][i1], B.x[sx][i2]};
      const double f = W[t] * PSI[t] * enr_weight(nef, v, xi);
      s += k < nef ? f * PSI[t] * enr_weight(nef, k, xi) : f * P[((size_t)e * npts + t) * 3 + (k - nef)];
    }
    if (k < nef) A[(size_t)(n3 + v) * N + n3 + k] = s;
    else R[(k - nef) * N + n3 + v] = s;
  }
  __syncthreads();
  // 6. Cholesky A = L L^T (lower triangle, right-looking); one warp per trailing row
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int j = 0; j < Nc; ++j) {
    const double d = A[(size_t)j * N + j];
    if (!(d > 0.0)) {
      if (tid == 0) atomicCAS(err, 0, c + 1);
      return;   // uniform: every thread read the same pivot after the barrier
    }
    const double ljj = sqrt(d);
    for (int i = j + 1 + tid; i < Nc; i += nt) {
      const double l = A[(size_t)i * N + j] / ljj;
      col[i] = l;
      A[(size_t)i * N + j] = l;
    }
    __syncthreads();
    if (tid == 0) A[(size_t)j * N + j] = ljj;
    for (int i = j + 1 + warp; i < Nc; i += nw) {
      const double li = col[i];
      for (int k = j + 1 + lane; k <= i; k += 32) A[(size_t)i * N + k] -= li * col[k];
    }
    __syncthreads();
  }
  if (!rhs) return;
  // 7. L y = r, then L^T x = y, for the three components
  for (int j = 0; j < Nc; ++j) {
    const double ljj = A[(size_t)j * N + j];
    if (tid < 3) R[tid * N + j] /= ljj;
    __syncthreads();
    for (int p = tid; p < 3 * (Nc - j - 1); p += nt) {
      const int a = p / (Nc - j - 1), i = j + 1 + p % (Nc - j - 1);
      R[a * N + i] -= A[(size_t)i * N + j] * R[a * N + j];
    }
    __syncthreads();
  }
  for (int j = Nc - 1; j >= 0; --j) {
    const double ljj = A[(size_t)j * N + j];
    if (tid < 3) R[tid * N + j] /= ljj;
    __syncthreads();
    for (int p = tid; p < 3 * j; p += nt) {
      const int a = p / j, i = p % j;
      R[a * N + i] -= A[(size_t)j * N + i] * R[a * N + j];
    }
    __syncthreads();
  }
  // 8. the cell's new coefficients
  for (int p = tid; p < 3 * n3; p += nt) {
    const int a = p / n3, i = p % n3;
    u_new[((size_t)c * 3 + a) * n3 + i] = R[a * N + i];
  }
  for (int p = tid; p < 3 * m.nef; p += nt) {
    const int a = p / m.nef, v = p % m.nef;
    u_new[3 * m.np + ((size_t)e * 3 + a) * m.nef + v] = nef ? R[a * N + n3 + v] : 0.0;
  }
}

// x = M^-1 r in the cells with the wall model switched on, from the Cholesky factor of the cell
// mass matrix in Ag (one CTA per enriched cell; the other cells are left untouched)
__global__ void chol_solve_kernel(MeshView<double> m, const int *__restrict__ enr_cell, const double *__restrict__ Ag,
                                  const double *__restrict__ r, double *__restrict__ x) {
  extern __shared__ double R[];
  const int e = blockIdx.x, c = enr_cell[e], tid = threadIdx.x, nt = blockDim.x;
  if (m.enr[c] < 0) return;
  const int n = m.n1, n3 = n * n * n, nef = m.nef, N = n3 + nef;
  const double *A = Ag + (size_t)e * N * N;
  for (int p = tid; p < 3 * N; p += nt) {
    const int a = p / N, i = p % N;
    R[p] = i < n3 ? r[((size_t)c * 3 + a) * n3 + i] : r[3 * m.np + ((size_t)e * 3 + a) * nef + (i - n3)];
  }
  __syncthreads();
  for (int j = 0; j < N; ++j) {
    if (tid < 3) R[tid * N + j] /= A[(size_t)j * N + j];
    __syncthreads();
    for (int p = tid; p < 3 * (N - j - 1); p += nt) {
      const int a = p / (N - j - 1), i = j + 1 + p % (N - j - 1);
      R[a * N + i] -= A[(size_t)i * N + j] * R[a * N + j];
    }
    __syncthreads();
  }
  for (int j = N - 1; j >= 0; --j) {
    if (tid < 3) R[tid * N + j] /= A[(size_t)j * N + j];
    __syncthreads();
    for (int p = tid; p < 3 * j; p += nt) {
      const int a = p / j, i = p % j;
      R[a * N + i] -= A[(size_t)j * N + i] * R[a * N + j];
    }
    __syncthreads();
  }
  for (int p = tid; p < 3 * N; p += nt) {
    const int a = p / N, i = p % N;
    if (i < n3) x[((size_t)c * 3 + a) * n3 + i] = R[p];
    else x[3 * m.np + ((size_t)e * 3 + a) * nef + (i - n3)] = R[p];
  }
}

}  // namespace

static cudaError_t proj_scratch(dgw_mesh *M, int nvec) {
  const int n = M->n1, N = n * n * n + M->nef;
  const int qx = M->basis64.q[M->P.full_quadrature ? QSET_WALL : QSET_LIN];
  const int npts = qx * M->basis64.q[QSET_WALL] * qx;
  cudaError_t e = cudaSuccess;
  if (!M->proj_A) {
    void *a = nullptr, *w = nullptr;
    e = cudaMalloc(&a, (size_t)M->ne * N * N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w, sizeof(int));
    for (void *q : {a, w})
      if (q) M->allocs.push_back(q);
    if (e != cudaSuccess) return e;
    M->hbm_bytes += (size_t)M->ne * N * N * sizeof(double) + sizeof(int);
    M->proj_A = (double *)a;
    M->proj_err = (int *)w;
  }
  if (M->proj_nvec < nvec) {
    void *p = nullptr;
    e = cudaMalloc(&p, (size_t)nvec * M->ne * npts * 3 * sizeof(double));
    if (e != cudaSuccess) return e;
    M->allocs.push_back(p);
    M->hbm_bytes += (size_t)nvec * M->ne * npts * 3 * sizeof(double);
    M->proj_P = (double *)p;
    M->proj_nvec = nvec;
  }
  return e;
}

cudaError_t launch_inverse_mass_cells(dgw_mesh *M, const double *r, double *x, cudaStream_t s) {
  if (M->ne == 0) return cudaSuccess;
  cudaError_t e = proj_scratch(M, 1);
  if (e != cudaSuccess) return e;
  const int n = M->n1, N = n * n * n + M->nef;
  const int q0 = M->basis64.q[M->P.full_quadrature ? QSET_WALL : QSET_LIN], q1 = M->basis64.q[QSET_WALL];
  if (!M->mass_factor_valid) {
    const ProjLayout L = proj_layout(n, q0, q1, M->nef);
    const size_t smem = (size_t)L.total * sizeof(double);
    e = cudaFuncSetAttribute(project_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->proj_err, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    note_launch();
    project_solve_kernel<<<M->ne, 256, smem, s>>>(M->v64, M->enr_cell_dev, M->v64.wt_vol[0], M->v64.nvol[0], nullptr,
                                                  M->proj_A, nullptr, M->proj_err);
    int h = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, M->proj_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (h) return cudaErrorInvalidValue;   // a cell mass matrix is not numerically positive definite
    M->mass_factor_valid = true;
  }
  note_launch();
  chol_solve_kernel<<<M->ne, 128, (size_t)3 * N * sizeof(double), s>>>(M->v64, M->enr_cell_dev, M->proj_A, r, x);
  return cudaGetLastError();
}

cudaError_t launch_projection(dgw_mesh *M, const double *tau_new, int nvec, const double *const *u_old,
                              double *const *u_new, cudaStream_t s, int *bad_cell) {
  *bad_cell = -1;
  const int n = M->n1;
  const int q0 = M->basis64.q[M->P.full_quadrature ? QSET_WALL : QSET_LIN], q1 = M->basis64.q[QSET_WALL], npts = q0 * q1 * q0;
  cudaError_t e = M->ne > 0 ? proj_scratch(M, nvec) : cudaSuccess;
  const size_t pstride = (size_t)M->ne * npts * 3;
  // every vector is evaluated in the old space before the tables change
  for (int v = 0; v < nvec && e == cudaSuccess && M->ne > 0; ++v) {
    note_launch();
    project_eval_kernel<<<M->ne, 128, 0, s>>>(M->v64, M->enr_cell_dev, u_old[v], M->v64.wt_vol[0], M->v64.nvol[0],
                                              M->proj_P + v * pstride);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_set_tau_nodes(M, tau_new, s);
  for (int v = 0; v < nvec && e == cudaSuccess; ++v)
    if (u_new[v] != u_old[v]) e = cudaMemcpyAsync(u_new[v], u_old[v], M->nu * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess || M->ne == 0) return e;
  const ProjLayout L = proj_layout(n, q0, q1, M->nef);
  const size_t smem = (size_t)L.total * sizeof(double);
  e = cudaFuncSetAttribute(project_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaMemsetAsync(M->proj_err, 0, sizeof(int), s);
  for (int v = 0; v < nvec && e == cudaSuccess; ++v) {
    note_launch();
    project_solve_kernel<<<M->ne, 256, smem, s>>>(M->v64, M->enr_cell_dev, M->v64.wt_vol[0], M->v64.nvol[0],
                                                  M->proj_P + v * pstride, M->proj_A, u_new[v], M->proj_err);
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, M->proj_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && h) *bad_cell = h - 1;
  // the last factorisation is that of the new space: the inverse mass can reuse it
  if (e == cudaSuccess && !h) M->mass_factor_valid = true;
  return e;
}

}  // namespace dgw
