// SIPG Laplacian on the channel of boxes, specialised by degree (Sec. 4.2 eq. ipflux, Sec. 4.4
// sum factorisation).
//
// On an axis-aligned box cell with exact Gauss integration, the cell and face integrals of the
// SIPG form factorise per direction: with the 1-D reference mass matrix M,
//   y_c = sum_d (L_d (x)_d M (x) M) u_c + sum_{d,s} (N_{d,s} (x)_d M (x) M) u_{nb(d,s)},
// where L_d (n x n) holds the stiffness along d plus the own-side face terms of both faces
// normal to d, and N_{d,s} is the rank-2 coupling to the neighbour across face s, which only
// needs the neighbour's trace value tv and reference normal derivative td on the shared face.
// With the 1-D stiffness K and the end derivatives D_s = l'(s), one line of L_d u + N u_nb is
//   out_a = a_d (K u)_a + sum_s [ p_s D_s,a (tv_s - u_e(s)) + delta_{a,e(s)} (-p_s D_s.u
//           + t_s (u_e(s) - tv_s) - e_s td_s) ],
// e(0) = 0, e(1) = k: the row of the cell (graded spacing, penalty) enters through seven scalars
// per direction (a_d = |K|/h_d^2, p_s = a_d sigma_s/2, t_s = |K| tau_s/h_d, e_s = |K| sigma_s/(2 h_d h'_d),
// zero for wall faces), while K, M and D_s depend only on the degree and sit in constant memory,
// so the fully unrolled line passes read them as instruction operands.
//
// Evaluation: y = M_z [ M_y (L_x u + nbr_x) + L_y (M_x u) + nbr_y' ] + L_z (M_x M_y u) + nbr_z'',
// three line passes (one thread owns a whole 1-D line in registers), with the y-face traces
// transformed by M_x and the z-face traces by M_x M_y. A CTA holds cpb consecutive cells along x.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "df64.cuh"
#include "sumfac.cuh"

namespace dgw {

// Per-row scalars: for d in {x, y, z}: a_d, p_0, p_1, t_0, t_1, e_0, e_1, (pad).
constexpr int kRowScal = 24;

// Degree tables: 1-D stiffness K, mass M (n x n, row-major), end derivatives D_0, D_1.
template <typename T>
struct BoxConst {
  T K[NMAX * NMAX];
  T M[NMAX * NMAX];
  T D[2][NMAX];
};
__constant__ BoxConst<float> c_box32[5];
__constant__ BoxConst<double> c_box64[5];
__constant__ BoxConst<df64> c_boxdf[5];   // double-float copies for the FP64-accurate FP32-pipe path

template <typename T>
__device__ __forceinline__ const BoxConst<T> &box_const(int k);
template <>
__device__ __forceinline__ const BoxConst<float> &box_const<float>(int k) { return c_box32[k - 1]; }
template <>
__device__ __forceinline__ const BoxConst<double> &box_const<double>(int k) { return c_box64[k - 1]; }
template <>
__device__ __forceinline__ const BoxConst<df64> &box_const<df64>(int k) { return c_boxdf[k - 1]; }

// FP32: up to 3 CTAs of <= 256 threads per SM for k <= 4 (register budget ~85/thread), 2 for k = 5;
// FP64 is FP64-pipe bound and keeps the default budget; double-float (two registers per value,
// about fifteen instructions per multiply-add) keeps two CTAs per SM.
template <typename T, int K>
struct BoxOcc { static constexpr int min_blocks = 1; };
template <int K>
struct BoxOcc<float, K> { static constexpr int min_blocks = K <= 4 ? 3 : 2; };
template <int K>
struct BoxOcc<df64, K> { static constexpr int min_blocks = 2; };

// One line of L_d u + N_d (tv, td) (see the file comment); R = the 8 scalars of direction d.
template <typename T, int K>
__device__ __forceinline__ void line_op(const T (&u)[K + 1], const T *R, T tv0, T td0, T tv1, T td1, T (&out)[K + 1]) {
  constexpr int n = K + 1;
  const BoxConst<T> &C = box_const<T>(K);
  const T a = R[0], p0 = R[1], p1 = R[2], t0 = R[3], t1 = R[4], e0 = R[5], e1 = R[6];
  const T j0 = tv0 - u[0], j1 = tv1 - u[n - 1];
  T d0 = r_zero<T>(), d1 = r_zero<T>();
#pragma unroll
  for (int b = 0; b < n; ++b) {
    d0 = r_fma(C.D[0][b], u[b], d0);
    d1 = r_fma(C.D[1][b], u[b], d1);
  }
  const T q0 = p0 * j0, q1 = p1 * j1;
#pragma unroll
  for (int r = 0; r < n; ++r) {
    T s = r_zero<T>();
#pragma unroll
    for (int b = 0; b < n; ++b) s = r_fma(C.K[r * n + b], u[b], s);
    out[r] = r_fma(C.D[1][r], q1, r_fma(C.D[0][r], q0, a * s));
  }
  out[0] = out[0] - r_fma(p0, d0, r_fma(t0, j0, e0 * td0));
  out[n - 1] = out[n - 1] - r_fma(p1, d1, r_fma(t1, j1, e1 * td1));
}

// v <- M v along a line of n values
template <typename T, int K>
__device__ __forceinline__ void mass_line(const T (&v)[K + 1], T (&out)[K + 1]) {
  constexpr int n = K + 1;
  const BoxConst<T> &C = box_const<T>(K);
#pragma unroll
  for (int r = 0; r < n; ++r) {
    T s = r_zero<T>();
#pragma unroll
    for (int b = 0; b < n; ++b) s = r_fma(C.M[r * n + b], v[b], s);
    out[r] = s;
  }
}

// T: storage type of p and y; R: compute type (T itself, or df64 for FP64-accurate arithmetic on the
// FP32 units with double vectors; that variant supports the plain epilogue only).
template <typename T, typename R, int K>
__global__ void __launch_bounds__(256, (BoxOcc<R, K>::min_blocks)) laplace_box_kernel(MeshView<T> m, const T *__restrict__ p,
                                                                                T *__restrict__ y, int cpb,
                                                                                LapEpi<T> epi) {
  constexpr int n = K + 1, n2 = n * n, n3 = n2 * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *Rs = reinterpret_cast<R *>(smem_raw);     // kRowScal
  R *U = Rs + kRowScal;                         // cpb n3 (input, then output)
  R *A = U + cpb * n3;                          // cpb n3 (T1 -> W)
  R *B = A + cpb * n3;                          // cpb n3 (T2 -> T3)
  R *TR = B + cpb * n3;                         // cpb * 6 faces * 2 (val, der) * n2
  R *TY = TR + cpb * 24 * n2;                   // cpb * 2 faces * 2 * n2 : y-face traces after M_x
  R *TZ = TY + cpb * 8 * n2;                    // cpb * 2 * 2 * n2 : z-face traces after M_x
  const BoxConst<R> &C = box_const<R>(K);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int c0 = blockIdx.x * cpb;
  if (blockIdx.y > 0) {   // column blockIdx.y of a block of vectors (the diagonal dinv is shared)
    const size_t co = (size_t)blockIdx.y * m.np;
    p += co;
    if (y) y += co;
    if (epi.b) epi.b += co;
    if (epi.d) epi.d += co;
    if (epi.xout) epi.xout += co;
  }
  const int i0 = c0 % m.nx, j = (c0 / m.nx) % m.ny, kz = c0 / (m.nx * m.ny);
  const T *Rg = m.rowops + (size_t)j * kRowScal;
  for (int t = tid; t < kRowScal; t += nt) Rs[t] = r_load<R>(Rg[t]);
  const T *pc = p + (size_t)c0 * n3;
  for (int t = tid; t < cpb * n3; t += nt) U[t] = r_load<R>(pc[t]);
  // Every thread owns line l of cell cl in all three passes (x-, y- then z-lines; l indexes the
  // face nodes of the same two tangential axes), so the index arithmetic is done once here.
  const bool line = tid < cpb * n2;
  const int cl = line ? tid / n2 : 0, l = line ? tid - cl * n2 : 0;
  const int lq = l / n, lr = l - lq * n;   // l = lr + n * lq
  int *nbr = reinterpret_cast<int *>(TZ + cpb * 8 * n2);   // [cpb][6] neighbour cells (-1: wall)
  if (tid < cpb * 6) {
    const int c = tid / 6, f = tid - c * 6, d = f >> 1, sg = (f & 1) ? 1 : -1;
    int ii = i0 + c, jj = j, kk = kz;
    if (d == 0) ii = (ii + sg + m.nx) % m.nx;
    else if (d == 2) kk = (kk + sg + m.nz) % m.nz;
    else jj += sg;
    nbr[tid] = (jj < 0 || jj >= m.ny) ? -1 : ii + m.nx * (jj + m.ny * kk);
  }
  __syncthreads();
  // neighbour traces at face node l of the six faces: value and reference normal derivative
  if (line) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1, side = f & 1, nb = nbr[cl * 6 + f];
      R val = r_zero<R>(), der = r_zero<R>();
      if (nb >= 0) {
        // neighbour endpoint on the shared face: side 0 -> its xi_d = 1, side 1 -> its xi_d = 0
        const int stride = d == 0 ? 1 : (d == 1 ? n : n2);
        const int base = d == 0 ? n * l : (d == 1 ? lr + n2 * lq : l);
        R v[n];
        // x-neighbours inside this CTA's row segment are already in shared memory
        if (nb >= c0 && nb < c0 + cpb) {
          const R *pn = U + (nb - c0) * n3;
#pragma unroll
          for (int b = 0; b < n; ++b) v[b] = pn[base + b * stride];
        } else {
          const T *pn = p + (size_t)nb * n3;
#pragma unroll
          for (int b = 0; b < n; ++b) v[b] = r_load<R>(pn[base + b * stride]);
        }
        val = side ? v[0] : v[n - 1];
#pragma unroll
        for (int b = 0; b < n; ++b) der = r_fma(side ? C.D[0][b] : C.D[1][b], v[b], der);
      }
      TR[((cl * 6 + f) * 2 + 0) * n2 + l] = val;
      TR[((cl * 6 + f) * 2 + 1) * n2 + l] = der;
    }
  }
  __syncthreads();
  // ---- phase A: x-lines (T1 = Lx u + nbr_x, T2 = M_x u); y- and z-traces <- M_x (items
  // it = l, l + n^2, ... < 4n: face (it / n) >> 1, array (it / n) & 1, t2 = it % n)
  if (line) {
    const int base = cl * n3 + n * l;
    R u[n], o1[n], o2[n];
#pragma unroll
    for (int b = 0; b < n; ++b) u[b] = U[base + b];
    const R v0 = TR[((cl * 6 + 0) * 2 + 0) * n2 + l], d0 = TR[((cl * 6 + 0) * 2 + 1) * n2 + l];
    const R v1 = TR[((cl * 6 + 1) * 2 + 0) * n2 + l], d1 = TR[((cl * 6 + 1) * 2 + 1) * n2 + l];
    line_op<R, K>(u, Rs, v0, d0, v1, d1, o1);
    mass_line<R, K>(u, o2);
#pragma unroll
    for (int a = 0; a < n; ++a) { A[base + a] = o1[a]; B[base + a] = o2[a]; }
    for (int it = l; it < 4 * n; it += n2) {   // one item per thread for k >= 3
      const int iq = it / n, ir = it - iq * n;
      const int fl = iq >> 1, arr = iq & 1;
#pragma unroll
      for (int isz = 0; isz < 2; ++isz) {
        const R *src = TR + ((cl * 6 + (isz ? 4 : 2) + fl) * 2 + arr) * n2 + n * ir;
        R *dst = (isz ? TZ : TY) + ((cl * 2 + fl) * 2 + arr) * n2 + n * ir;
        R v[n], o[n];
#pragma unroll
        for (int b = 0; b < n; ++b) v[b] = src[b];
        mass_line<R, K>(v, o);
#pragma unroll
        for (int a = 0; a < n; ++a) dst[a] = o[a];
      }
    }
  }
  __syncthreads();
  // ---- phase B: y-lines at (x, z) = (lr, lq): W = M_y T1 + Ly T2 + nbr_y', T3 = M_y T2; z-face
  // traces (indexed x + n*y) <- M_y (items it as in phase A, x = it % n)
  if (line) {
    const int base = cl * n3 + lr + n2 * lq;
    R a1[n], a2[n], w[n], t3[n], ly[n];
#pragma unroll
    for (int c = 0; c < n; ++c) { a1[c] = A[base + n * c]; a2[c] = B[base + n * c]; }
    const R v0 = TY[((cl * 2 + 0) * 2 + 0) * n2 + l], d0 = TY[((cl * 2 + 0) * 2 + 1) * n2 + l];
    const R v1 = TY[((cl * 2 + 1) * 2 + 0) * n2 + l], d1 = TY[((cl * 2 + 1) * 2 + 1) * n2 + l];
    line_op<R, K>(a2, Rs + 8, v0, d0, v1, d1, ly);
    mass_line<R, K>(a1, w);
    mass_line<R, K>(a2, t3);
#pragma unroll
    for (int b = 0; b < n; ++b) { A[base + n * b] = w[b] + ly[b]; B[base + n * b] = t3[b]; }
    for (int it = l; it < 4 * n; it += n2) {
      const int iq = it / n, ir = it - iq * n;
      const int fl = iq >> 1, arr = iq & 1;
      const R *src = TZ + ((cl * 2 + fl) * 2 + arr) * n2 + ir;
      R *dst = TR + ((cl * 6 + 4 + fl) * 2 + arr) * n2 + ir;
      R v[n], o[n];
#pragma unroll
      for (int b = 0; b < n; ++b) v[b] = src[n * b];
      mass_line<R, K>(v, o);
#pragma unroll
      for (int a = 0; a < n; ++a) dst[n * a] = o[a];
    }
  }
  __syncthreads();
  // ---- phase C: z-lines at l = x + n*y (y = M_z W + Lz T3 + nbr_z'')
  if (line) {
    const int base = cl * n3 + l;
    R a1[n], a2[n], w[n], lz[n];
#pragma unroll
    for (int e = 0; e < n; ++e) { a1[e] = A[base + n2 * e]; a2[e] = B[base + n2 * e]; }
    const R v0 = TR[((cl * 6 + 4) * 2 + 0) * n2 + l], d0 = TR[((cl * 6 + 4) * 2 + 1) * n2 + l];
    const R v1 = TR[((cl * 6 + 5) * 2 + 0) * n2 + l], d1 = TR[((cl * 6 + 5) * 2 + 1) * n2 + l];
    line_op<R, K>(a2, Rs + 16, v0, d0, v1, d1, lz);
    mass_line<R, K>(a1, w);
#pragma unroll
    for (int c = 0; c < n; ++c) U[base + n2 * c] = w[c] + lz[c];
  }
  __syncthreads();
  const size_t o = (size_t)c0 * n3;
  if (epi.mode == LAP_PLAIN) {
    for (int t = tid; t < cpb * n3; t += nt) y[o + t] = r_store<T>(U[t]);
  } else if constexpr (std::is_same<T, R>::value) {
    if (epi.mode == LAP_RESIDUAL) {
      for (int t = tid; t < cpb * n3; t += nt) y[o + t] = epi.b[o + t] - U[t];
    } else {
      for (int t = tid; t < cpb * n3; t += nt) {
        const size_t i = o + t;
        const T dn = (epi.first ? T(0) : epi.c1 * epi.d[i]) + epi.c2 * epi.dinv[i] * (epi.b[i] - U[t]);
        epi.d[i] = dn;
        epi.xout[i] = p[i] + dn;
      }
    }
  }
}

template <typename T>
static size_t box_smem(int n, int cpb) {
  const int n2 = n * n, n3 = n2 * n;
  return sizeof(T) * ((size_t)kRowScal + 3 * (size_t)cpb * n3 + (size_t)cpb * (24 + 8 + 8) * n2) +
         sizeof(int) * (size_t)cpb * 6;
}

// cells per CTA: the largest power of two dividing nx with cpb*(k+1)^2 <= 256 and cpb <= 8
static int box_cpb(int nx, int n) {
  int c = 1;
  while (c * 2 <= 8 && (c * 2) * n * n <= 256 && nx % (c * 2) == 0) c *= 2;
  return c;
}

// Degree tables in constant memory, written once per device before the first box kernel runs.
cudaError_t box_constants_init() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
  BoxConst<double> h64[5];
  BoxConst<float> h32[5];
  std::memset(h64, 0, sizeof(h64));
  std::memset(h32, 0, sizeof(h32));
  for (int k = 1; k <= 5; ++k) {
    Basis<double> B;
    fill_basis<double>(k, k + 1, k + 1, &B);
    const int n = k + 1, q = B.q[QSET_LIN];
    for (int a = 0; a < n; ++a) {
      for (int b = 0; b < n; ++b) {
        double mv = 0.0, kv = 0.0;
        for (int t = 0; t < q; ++t) {
          mv += B.w[QSET_LIN][t] * B.S[QSET_LIN][t * n + a] * B.S[QSET_LIN][t * n + b];
          kv += B.w[QSET_LIN][t] * B.D[QSET_LIN][t * n + a] * B.D[QSET_LIN][t * n + b];
        }
        h64[k - 1].M[a * n + b] = mv;
        h64[k - 1].K[a * n + b] = kv;
      }
      h64[k - 1].D[0][a] = B.dend[0][a];
      h64[k - 1].D[1][a] = B.dend[1][a];
    }
    for (int i = 0; i < NMAX * NMAX; ++i) {
      h32[k - 1].M[i] = (float)h64[k - 1].M[i];
      h32[k - 1].K[i] = (float)h64[k - 1].K[i];
    }
    for (int sd = 0; sd < 2; ++sd)
      for (int i = 0; i < NMAX; ++i) h32[k - 1].D[sd][i] = (float)h64[k - 1].D[sd][i];
  }
  // double-float copies: hi = nearest float, lo = nearest float to the remainder
  BoxConst<df64> hdf[5];
  std::memset(hdf, 0, sizeof(hdf));
  auto split = [](double v) { const float h = (float)v; return df64{h, (float)(v - (double)h)}; };
  for (int k = 0; k < 5; ++k) {
    for (int i = 0; i < NMAX * NMAX; ++i) {
      hdf[k].M[i] = split(h64[k].M[i]);
      hdf[k].K[i] = split(h64[k].K[i]);
    }
    for (int sd = 0; sd < 2; ++sd)
      for (int i = 0; i < NMAX; ++i) hdf[k].D[sd][i] = split(h64[k].D[sd][i]);
  }
  e = cudaMemcpyToSymbol(c_box64, h64, sizeof(h64));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_box32, h32, sizeof(h32));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_boxdf, hdf, sizeof(hdf));
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

template <typename T, typename R, int K>
static cudaError_t launch_box_k(const MeshView<T> &m, const T *p, T *y, const LapEpi<T> &epi, cudaStream_t s) {
  constexpr int n = K + 1;
  const int cpb = box_cpb(m.nx, n);
  const size_t sm = box_smem<R>(n, cpb);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(laplace_box_kernel<T, R, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e == cudaSuccess)   // the whole unified L1/shared array as shared memory: more CTAs per SM
      e = cudaFuncSetAttribute(laplace_box_kernel<T, R, K>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int threads = ((cpb * n * n + 31) / 32) * 32;
  const int ncols = epi.ncols > 1 ? epi.ncols : 1;
  note_launch();
  note_dofs(m.np * ncols);
  laplace_box_kernel<T, R, K><<<dim3(m.nc / cpb, ncols), threads, sm, s>>>(m, p, y, cpb, epi);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_laplace_epi(const MeshView<T> &m, const T *p, T *y, const LapEpi<T> &epi, cudaStream_t s) {
  if (epi.mode == LAP_CHEB && epi.xout == p) return cudaErrorInvalidValue;   // neighbours read p
  if (epi.ncols > 1 && m.geo == GEO_CURVED) return cudaErrorNotSupported;      // columns: boxes only
  if (m.geo == GEO_CURVED) {   // per-point metrics: the table-driven kernel, else the general one
    if (m.lvol && m.lface) return launch_curved_laplace<T>(m, p, y, epi, s);
    return launch_vector_op<T>(OP_LAP, m, p, y, s, &epi);
  }
  switch (m.n1) {
    case 2: return launch_box_k<T, T, 1>(m, p, y, epi, s);
    case 3: return launch_box_k<T, T, 2>(m, p, y, epi, s);
    case 4: return launch_box_k<T, T, 3>(m, p, y, epi, s);
    case 5: return launch_box_k<T, T, 4>(m, p, y, epi, s);
    case 6: return launch_box_k<T, T, 5>(m, p, y, epi, s);
  }
  return cudaErrorInvalidValue;
}

// y = A_L p with double vectors and double-float arithmetic (boxes only; plain epilogue)
cudaError_t launch_laplace_df(const MeshView<double> &m, const double *p, double *y, cudaStream_t s) {
  if (m.geo == GEO_CURVED) return cudaErrorNotSupported;
  LapEpi<double> epi{};
  epi.mode = LAP_PLAIN;
  switch (m.n1) {
    case 2: return launch_box_k<double, df64, 1>(m, p, y, epi, s);
    case 3: return launch_box_k<double, df64, 2>(m, p, y, epi, s);
    case 4: return launch_box_k<double, df64, 3>(m, p, y, epi, s);
    case 5: return launch_box_k<double, df64, 4>(m, p, y, epi, s);
    case 6: return launch_box_k<double, df64, 5>(m, p, y, epi, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_laplace(const MeshView<T> &m, const T *p, T *y, cudaStream_t s) {
  LapEpi<T> epi{};
  epi.mode = LAP_PLAIN;
  return launch_laplace_epi<T>(m, p, y, epi, s);
}

template cudaError_t launch_laplace<double>(const MeshView<double> &, const double *, double *, cudaStream_t);
template cudaError_t launch_laplace<float>(const MeshView<float> &, const float *, float *, cudaStream_t);
template cudaError_t launch_laplace_epi<double>(const MeshView<double> &, const double *, double *,
                                                const LapEpi<double> &, cudaStream_t);
template cudaError_t launch_laplace_epi<float>(const MeshView<float> &, const float *, float *, const LapEpi<float> &,
                                               cudaStream_t);

// Per-row scalars of the factorised operator (see the file comment): with h = (hx, hy_j, hz),
// |K| = hx hy hz, for direction d and face s present (g_s = 1; y-faces at the walls are absent):
// a_d = |K|/h_d^2, p_s = a_d sigma_s/2, t_s = |K| tau_s/h_d (tau_s: max over the two cells),
// e_s = |K| sigma_s/(2 h_d h'_d) (h'_d: the neighbour's spacing), sigma_0 = -1, sigma_1 = +1.
void box_rowscal(const BoxGeometry &g, std::vector<double> &R) {
  R.assign((size_t)g.ny * kRowScal, 0.0);
  for (int j = 0; j < g.ny; ++j) {
    double *Rj = R.data() + (size_t)j * kRowScal;
    const double h[3] = {g.hx, g.hy[j], g.hz};
    const double hV = h[0] * h[1] * h[2];
    const double tauc = g.tau[(size_t)j * g.nx];
    for (int d = 0; d < 3; ++d) {
      double *r = Rj + 8 * d;
      const double hd = h[d], sc = hV / hd;
      r[0] = sc / hd;
      for (int s = 0; s < 2; ++s) {
        double tau = tauc, hdo = hd;
        if (d == 1) {
          const int jn = j + (s ? 1 : -1);
          if (jn < 0 || jn >= g.ny) continue;   // homogeneous Neumann on walls: no face terms
          tau = std::max(tauc, g.tau[(size_t)jn * g.nx]);
          hdo = g.hy[jn];
        }
        const double sig = s ? 1.0 : -1.0;
        r[1 + s] = 0.5 * sig * sc / hd;
        r[3 + s] = sc * tau;
        r[5 + s] = 0.5 * sig * sc / hdo;
      }
    }
  }
}

// Full per-row 1-D operators of the same factorisation (host assembly of small coarse-level
// matrices): Lx, Ly, Lz (n*n each), then for d in {x,y,z}, s in {0,1}: c1[n], c2[n].
static constexpr int rowops_size(int n) { return 3 * n * n + 12 * n; }

// Per-row 1-D operators of the factorised SIPG Laplacian (see the file comment).
void box_rowops(const BoxGeometry &g, const Basis<double> &B, std::vector<double> &R) {
  const int n = g.k + 1, n2 = n * n, ROW = rowops_size(n);
  std::vector<double> M(n2, 0.0), K(n2, 0.0);
  const int q = B.q[QSET_LIN];
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int t = 0; t < q; ++t) {
        M[a * n + b] += B.w[QSET_LIN][t] * B.S[QSET_LIN][t * n + a] * B.S[QSET_LIN][t * n + b];
        K[a * n + b] += B.w[QSET_LIN][t] * B.D[QSET_LIN][t * n + a] * B.D[QSET_LIN][t * n + b];
      }
  R.assign((size_t)g.ny * ROW, 0.0);
  for (int j = 0; j < g.ny; ++j) {
    double *Rj = R.data() + (size_t)j * ROW;
    const double h[3] = {g.hx, g.hy[j], g.hz};
    const double hV = h[0] * h[1] * h[2];
    const double tauc = g.tau[(size_t)j * g.nx];
    for (int d = 0; d < 3; ++d) {
      double *L = Rj + d * n2;
      const double hd = h[d], sc = hV / hd;
      for (int t = 0; t < n2; ++t) L[t] = sc * K[t] / hd;
      for (int s = 0; s < 2; ++s) {
        bool has = true;
        double tau = tauc, hdo = hd;
        if (d == 1) {
          const int jn = j + (s ? 1 : -1);
          has = jn >= 0 && jn < g.ny;
          if (has) { tau = std::max(tauc, g.tau[(size_t)jn * g.nx]); hdo = g.hy[jn]; }
        }
        double *c1 = Rj + 3 * n2 + (d * 2 + s) * 2 * n, *c2 = c1 + n;
        if (!has) continue;   // homogeneous Neumann on walls: no face terms
        const double sig = s ? 1.0 : -1.0;
        const int end = s ? n - 1 : 0;
        const double *Ds = B.dend[s];
        // own-side face terms
        for (int a = 0; a < n; ++a)
          for (int b = 0; b < n; ++b) {
            double v = -0.5 * (sig / hd) * (Ds[a] * (b == end) + (a == end) * Ds[b]);
            if (a == end && b == end) v += tau;
            L[a * n + b] += sc * v;
          }
        // neighbour coupling: c1 (x) trace value + c2 (x) trace reference derivative
        for (int a = 0; a < n; ++a) {
          c1[a] = sc * (0.5 * (sig / hd) * Ds[a] - (a == end ? tau : 0.0));
          c2[a] = sc * (a == end ? -0.5 * sig / hdo : 0.0);
        }
      }
    }
  }
}

// Host reference of the same factorised operator (assembles small coarse-level matrices).
void host_box_apply(const BoxGeometry &g, const Basis<double> &B, const std::vector<double> &R, const double *x,
                    double *y) {
  const int n = g.k + 1, n2 = n * n, n3 = n2 * n, ROW = rowops_size(n);
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  std::vector<double> v(n3), w(n3);
  auto idx = [&](int d, int a, int t1, int t2) {   // local index with coordinate a along d
    int c[3];
    const int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
    c[d] = a; c[o1] = t1; c[o2] = t2;
    return c[0] + n * (c[1] + n * c[2]);
  };
  for (int kz = 0; kz < nz; ++kz)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t c = i + (size_t)nx * (j + (size_t)ny * kz);
        const double *u = x + c * n3;
        const double *Rj = R.data() + (size_t)j * ROW;
        double *yc = y + c * n3;
        for (int t = 0; t < n3; ++t) yc[t] = 0.0;
        for (int d = 0; d < 3; ++d) {
          const double *L = Rj + d * n2;
          for (int t2 = 0; t2 < n; ++t2)
            for (int t1 = 0; t1 < n; ++t1)
              for (int a = 0; a < n; ++a) {
                double sum = 0.0;
                for (int b = 0; b < n; ++b) sum += L[a * n + b] * u[idx(d, b, t1, t2)];
                v[idx(d, a, t1, t2)] = sum;
              }
          for (int sd = 0; sd < 2; ++sd) {
            int ii = i, jj = j, kk = kz;
            const int sg = sd ? 1 : -1;
            if (d == 0) ii = (i + sg + nx) % nx;
            else if (d == 2) kk = (kz + sg + nz) % nz;
            else { jj = j + sg; if (jj < 0 || jj >= ny) continue; }
            const double *un = x + (ii + (size_t)nx * (jj + (size_t)ny * kk)) * n3;
            const double *c1 = Rj + 3 * n2 + (d * 2 + sd) * 2 * n, *c2 = c1 + n;
            const int ep = sd ? 0 : 1, lay = ep ? n - 1 : 0;
            for (int t2 = 0; t2 < n; ++t2)
              for (int t1 = 0; t1 < n; ++t1) {
                const double tv = un[idx(d, lay, t1, t2)];
                double td = 0.0;
                for (int b = 0; b < n; ++b) td += B.dend[ep][b] * un[idx(d, b, t1, t2)];
                for (int a = 0; a < n; ++a) v[idx(d, a, t1, t2)] += c1[a] * tv + c2[a] * td;
              }
          }
          // M along the two other directions
          for (int e = 0; e < 3; ++e) {
            if (e == d) continue;
            for (int t2 = 0; t2 < n; ++t2)
              for (int t1 = 0; t1 < n; ++t1)
                for (int a = 0; a < n; ++a) {
                  double sum = 0.0;
                  for (int b = 0; b < n; ++b) sum += B.mass[a * n + b] * v[idx(e, b, t1, t2)];
                  w[idx(e, a, t1, t2)] = sum;
                }
            v.swap(w);
          }
          for (int t = 0; t < n3; ++t) yc[t] += v[t];
        }
      }
}

}  // namespace dgw
