// SIPG Laplacian (eq. ipflux) on curved cells, specialised by degree: the same weak form as the
// general operator kernel (OP_LAP in ops.cu) evaluated from two per-column tables,
//   lvol  = |det J| w J^-1 J^-T at the (k+1)^3 Gauss points (cell term grad phi . G grad u), and
//   lface = dA, dA J^-1 n (own side), dA J^-1 n (neighbour at the shared point) at the face points,
// so a reference gradient dotted with J^-1 n gives the normal derivative times the area weight.
//
// A CTA holds cpb cells of one row segment; every thread owns one line of one cell in each line
// pass and keeps it in registers. Volume: x-, y- then z-lines take u to the reference gradient at
// the Gauss points; the z pass also applies G and the first transposed pass; then y- and x-lines
// integrate back. Faces: while owning a d-line a thread extracts the face layer and the reference
// normal derivative on both faces normal to d, for the cell and for its neighbour (whose line is
// read from global memory, or from shared memory inside the row segment); two tangential passes
// give value and reference gradient of both sides at the face points, the flux coefficients of
// the test functions follow pointwise, two transposed passes return them to the face nodes, and the
// x-line owners add them (layer value and l'(side)-weighted normal derivative) to their nodes.
// Seven barriers per CTA.
#include <cstring>
#include <mutex>

#include "metric.cuh"

namespace dgw {

// Degree tables: S[a*n+b] = l_b(x_a), D[a*n+b] = l_b'(x_a) at the k+1 Gauss points, E[s][b] = l_b'(s).
template <typename T>
struct CurvConst {
  T S[NMAX * NMAX];
  T D[NMAX * NMAX];
  T E[2][NMAX];
};
__constant__ CurvConst<float> c_curv32[5];
__constant__ CurvConst<double> c_curv64[5];

template <typename T>
__device__ __forceinline__ const CurvConst<T> &curv_const(int k);
template <>
__device__ __forceinline__ const CurvConst<float> &curv_const<float>(int k) { return c_curv32[k - 1]; }
template <>
__device__ __forceinline__ const CurvConst<double> &curv_const<double>(int k) { return c_curv64[k - 1]; }

cudaError_t curved_constants_init() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
  CurvConst<double> h64[5];
  CurvConst<float> h32[5];
  std::memset(h64, 0, sizeof(h64));
  std::memset(h32, 0, sizeof(h32));
  for (int k = 1; k <= 5; ++k) {
    Basis<double> B;
    fill_basis<double>(k, k + 1, k + 1, &B);
    const int n = k + 1;
    for (int i = 0; i < n * n; ++i) {
      h64[k - 1].S[i] = B.S[QSET_LIN][i];
      h64[k - 1].D[i] = B.D[QSET_LIN][i];
      h32[k - 1].S[i] = (float)B.S[QSET_LIN][i];
      h32[k - 1].D[i] = (float)B.D[QSET_LIN][i];
    }
    for (int sd = 0; sd < 2; ++sd)
      for (int b = 0; b < n; ++b) {
        h64[k - 1].E[sd][b] = B.dend[sd][b];
        h32[k - 1].E[sd][b] = (float)B.dend[sd][b];
      }
  }
  e = cudaMemcpyToSymbol(c_curv64, h64, sizeof(h64));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_curv32, h32, sizeof(h32));
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

// out_a = sum_b M[a*n+b] v_b (forward) or sum_b M[b*n+a] v_b (transposed)
template <typename T, int n, bool TR>
__device__ __forceinline__ void mat_line(const T *M, const T (&v)[n], T (&out)[n]) {
#pragma unroll
  for (int a = 0; a < n; ++a) {
    T s = T(0);
#pragma unroll
    for (int b = 0; b < n; ++b) s += (TR ? M[b * n + a] : M[a * n + b]) * v[b];
    out[a] = s;
  }
}

// Shared memory per cell (in T): U, X0, X1 (n^3 each), Y (3 n^3), LAY (24 n^2: face x {own val,
// own der, nb val, nb der} x node), AS (24 n^2), AD (12 n^2); the flux integrals I (18 n^2) reuse
// LAY and the face-node coefficients FL, GL (12 n^2) reuse AS.
template <int n>
struct CurvPlan {
  static constexpr int n2 = n * n, n3 = n2 * n;
  static constexpr int U = 0, X0 = n3, X1 = 2 * n3, Y = 3 * n3, LAY = 6 * n3, AS = LAY + 24 * n2,
                       AD = AS + 24 * n2, per_cell = AD + 12 * n2;
};

template <typename T, int K>
__global__ void __launch_bounds__(256) curved_laplace_kernel(MeshView<T> m, const T *__restrict__ p, T *__restrict__ y,
                                                            int cpb, LapEpi<T> epi) {
  constexpr int n = K + 1, n2 = n * n, n3 = n2 * n;
  using PL = CurvPlan<n>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  int *nbr = reinterpret_cast<int *>(sm + (size_t)cpb * PL::per_cell);   // [cpb][6]
  const CurvConst<T> &C = curv_const<T>(K);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int c0 = blockIdx.x * cpb;
  const int i0 = c0 % m.nx, j = (c0 / m.nx) % m.ny, kz = c0 / (m.nx * m.ny);
  for (int t = tid; t < cpb * n3; t += nt) {
    const int cl = t / n3;
    sm[cl * PL::per_cell + PL::U + (t - cl * n3)] = p[(size_t)c0 * n3 + t];
  }
  if (tid < cpb * 6) {
    const int c = tid / 6, f = tid - c * 6, d = f >> 1, sg = (f & 1) ? 1 : -1;
    int ii = i0 + c, jj = j, kk = kz;
    if (d == 0) ii = (ii + sg + m.nx) % m.nx;
    else if (d == 2) kk = (kk + sg + m.nz) % m.nz;
    else jj += sg;
    nbr[tid] = (jj < 0 || jj >= m.ny) ? -1 : ii + m.nx * (jj + m.ny * kk);
  }
  __syncthreads();
  const bool line = tid < cpb * n2;
  const int cl = line ? tid / n2 : 0, l = line ? tid - cl * n2 : 0;
  const int lq = l / n, lr = l - lq * n;   // l = lr + n lq
  T *cs = sm + cl * PL::per_cell;
  const int col = (i0 + cl) + m.nx * j;
  // face layers of the two faces normal to d seen by a thread owning the d-line at face node l:
  // own value / derivative from the cell's line u, neighbour's from its line on the far side
  auto layers = [&](int d, const T (&u)[n], int stride, int base) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int f = 2 * d + s;
      T *L = cs + PL::LAY + f * 4 * n2;
      T der = T(0);
#pragma unroll
      for (int b = 0; b < n; ++b) der += C.E[s][b] * u[b];
      L[l] = s ? u[n - 1] : u[0];
      L[n2 + l] = der;
      const int nb = nbr[cl * 6 + f];
      T vv = T(0), dv = T(0);
      if (nb >= 0) {
        const T *pn = (nb >= c0 && nb < c0 + cpb) ? sm + (nb - c0) * PL::per_cell + PL::U : p + (size_t)nb * n3;
        T v[n];
#pragma unroll
        for (int b = 0; b < n; ++b) v[b] = pn[base + b * stride];
        vv = s ? v[0] : v[n - 1];   // the neighbour's face at xi_d = 1 - s
#pragma unroll
        for (int b = 0; b < n; ++b) dv += C.E[1 - s][b] * v[b];
      }
      L[2 * n2 + l] = vv;
      L[3 * n2 + l] = dv;
    }
  };
  // ---- P1: x-lines at (y, z) = (lr, lq): X0 = S u, X1 = D u; x-face layers
  if (line) {
    T u[n], a[n], b[n];
#pragma unroll
    for (int t = 0; t < n; ++t) u[t] = cs[PL::U + n * l + t];
    mat_line<T, n, false>(C.S, u, a);
    mat_line<T, n, false>(C.D, u, b);
#pragma unroll
    for (int t = 0; t < n; ++t) { cs[PL::X0 + n * l + t] = a[t]; cs[PL::X1 + n * l + t] = b[t]; }
    layers(0, u, 1, n * l);
  }
  __syncthreads();
  // ---- P2: y-lines at (x, z) = (lr, lq): Y00 = S X0, Y01 = D X0, Y10 = S X1; y-face layers of u
  if (line) {
    const int base = lr + n2 * lq;
    T x0[n], x1[n], u[n], o[n];
#pragma unroll
    for (int t = 0; t < n; ++t) {
      x0[t] = cs[PL::X0 + base + n * t];
      x1[t] = cs[PL::X1 + base + n * t];
      u[t] = cs[PL::U + base + n * t];
    }
    mat_line<T, n, false>(C.S, x0, o);
#pragma unroll
    for (int t = 0; t < n; ++t) cs[PL::Y + base + n * t] = o[t];
    mat_line<T, n, false>(C.D, x0, o);
#pragma unroll
    for (int t = 0; t < n; ++t) cs[PL::Y + n3 + base + n * t] = o[t];
    mat_line<T, n, false>(C.S, x1, o);
#pragma unroll
    for (int t = 0; t < n; ++t) cs[PL::Y + 2 * n3 + base + n * t] = o[t];
    layers(1, u, n, base);
  }
  __syncthreads();
  // ---- P3: z-lines at (x, y) = (lr, lq): reference gradient, H = G g, transposed z pass
  // (Tx = S^T Hx, Ty = S^T Hy, Tz = D^T Hz, written over Y); z-face layers of u
  if (line) {
    const int base = l;
    T y00[n], y01[n], y10[n], u[n], gx[n], gy[n], gz[n];
#pragma unroll
    for (int t = 0; t < n; ++t) {
      y00[t] = cs[PL::Y + base + n2 * t];
      y01[t] = cs[PL::Y + n3 + base + n2 * t];
      y10[t] = cs[PL::Y + 2 * n3 + base + n2 * t];
      u[t] = cs[PL::U + base + n2 * t];
    }
    mat_line<T, n, false>(C.D, y00, gz);
    mat_line<T, n, false>(C.S, y01, gy);
    mat_line<T, n, false>(C.S, y10, gx);
    const T *G = m.lvol + ((size_t)col * n3 + base) * 6;
#pragma unroll
    for (int t = 0; t < n; ++t) {
      const T *g = G + (size_t)t * n2 * 6;
      const T hx = g[0] * gx[t] + g[3] * gy[t] + g[4] * gz[t];
      const T hy = g[3] * gx[t] + g[1] * gy[t] + g[5] * gz[t];
      const T hz = g[4] * gx[t] + g[5] * gy[t] + g[2] * gz[t];
      gx[t] = hx; gy[t] = hy; gz[t] = hz;
    }
    T o[n];
    mat_line<T, n, true>(C.S, gx, o);
#pragma unroll
    for (int t = 0; t < n; ++t) cs[PL::Y + base + n2 * t] = o[t];
    mat_line<T, n, true>(C.S, gy, o);
#pragma unroll
    for (int t = 0; t < n; ++t) cs[PL::Y + n3 + base + n2 * t] = o[t];
    mat_line<T, n, true>(C.D, gz, o);
#pragma unroll
    for (int t = 0; t < n; ++t) cs[PL::Y + 2 * n3 + base + n2 * t] = o[t];
    layers(2, u, n2, base);
  }
  __syncthreads();
  // ---- P4: y-lines: V0 = S^T Tx, V1 = D^T Ty + S^T Tz (into X0, X1); F1: face layers along t1
  if (line) {
    const int base = lr + n2 * lq;
    T tx[n], ty[n], tz[n], o[n], o2[n];
#pragma unroll
    for (int t = 0; t < n; ++t) {
      tx[t] = cs[PL::Y + base + n * t];
      ty[t] = cs[PL::Y + n3 + base + n * t];
      tz[t] = cs[PL::Y + 2 * n3 + base + n * t];
    }
    mat_line<T, n, true>(C.S, tx, o);
#pragma unroll
    for (int t = 0; t < n; ++t) cs[PL::X0 + base + n * t] = o[t];
    mat_line<T, n, true>(C.D, ty, o);
    mat_line<T, n, true>(C.S, tz, o2);
#pragma unroll
    for (int t = 0; t < n; ++t) cs[PL::X1 + base + n * t] = o[t] + o2[t];
  }
  // F1 items (cell c, face f, array k, node i2 along t2): S (and for values D) along t1
  for (int it = tid; it < cpb * 6 * 4 * n; it += nt) {
    const int c = it / (24 * n), r = it - c * 24 * n, f = r / (4 * n), k = (r / n) & 3, i2 = r % n;
    T *cc = sm + c * PL::per_cell;
    const T *src = cc + PL::LAY + (f * 4 + k) * n2 + n * i2;
    T v[n], o[n];
#pragma unroll
    for (int t = 0; t < n; ++t) v[t] = src[t];
    mat_line<T, n, false>(C.S, v, o);
#pragma unroll
    for (int a = 0; a < n; ++a) cc[PL::AS + (f * 4 + k) * n2 + a + n * i2] = o[a];   // [a1 + n i2]
    if ((k & 1) == 0) {
      mat_line<T, n, false>(C.D, v, o);
#pragma unroll
      for (int a = 0; a < n; ++a) cc[PL::AD + (f * 2 + (k >> 1)) * n2 + a + n * i2] = o[a];
    }
  }
  __syncthreads();
  // ---- F2: per (cell, face, point a1 along t1): both sides' value and reference gradient along t2,
  // flux coefficients of the own test functions, transposed pass along t2 into I (over LAY)
  for (int it = tid; it < cpb * 6 * n; it += nt) {
    const int c = it / (6 * n), r = it - c * 6 * n, f = r / n, a1 = r % n;
    T *cc = sm + c * PL::per_cell;
    T *I = cc + PL::LAY + f * 3 * n2;   // I0, I1, I2: [a1 + n i2]
    const int nb = nbr[c * 6 + f];
    if (nb < 0) {   // homogeneous Neumann wall: no face terms
#pragma unroll
      for (int t = 0; t < n; ++t) { I[a1 + n * t] = T(0); I[n2 + a1 + n * t] = T(0); I[2 * n2 + a1 + n * t] = T(0); }
      continue;
    }
    const int d = f >> 1, t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    T val[2][n], dd[2][n], dt1[2][n], dt2[2][n];
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      T av[n], ad[n], adr[n];
#pragma unroll
      for (int t = 0; t < n; ++t) {
        av[t] = cc[PL::AS + (f * 4 + 2 * sd) * n2 + a1 + n * t];
        adr[t] = cc[PL::AS + (f * 4 + 2 * sd + 1) * n2 + a1 + n * t];
        ad[t] = cc[PL::AD + (f * 2 + sd) * n2 + a1 + n * t];
      }
      mat_line<T, n, false>(C.S, av, val[sd]);
      mat_line<T, n, false>(C.D, av, dt2[sd]);
      mat_line<T, n, false>(C.S, ad, dt1[sd]);
      mat_line<T, n, false>(C.S, adr, dd[sd]);
    }
    const T tau = max(m.tau[c0 + c], m.tau[nb]);
    const T *F = m.lface + (((size_t)((i0 + c) + m.nx * j) * 6 + f) * n2 + a1) * 7;
    T c0v[n], cd[n], ct1[n], ct2[n];
#pragma unroll
    for (int a2 = 0; a2 < n; ++a2) {
      const T *g = F + (size_t)a2 * n * 7;
      const T gs[3] = {g[1], g[2], g[3]}, go[3] = {g[4], g[5], g[6]};
      T r0[3], r1[3];   // reference gradients of both sides, by reference axis
      r0[d] = dd[0][a2]; r0[t1] = dt1[0][a2]; r0[t2] = dt2[0][a2];
      r1[d] = dd[1][a2]; r1[t1] = dt1[1][a2]; r1[t2] = dt2[1][a2];
      const T dn = gs[0] * r0[0] + gs[1] * r0[1] + gs[2] * r0[2] + go[0] * r1[0] + go[1] * r1[1] + go[2] * r1[2];
      const T jump = val[0][a2] - val[1][a2];
      c0v[a2] = T(-0.5) * dn + tau * g[0] * jump;
      const T hj = T(-0.5) * jump;
      cd[a2] = hj * gs[d];
      ct1[a2] = hj * gs[t1];
      ct2[a2] = hj * gs[t2];
    }
    T o[n], o2[n];
    mat_line<T, n, true>(C.S, c0v, o);
    mat_line<T, n, true>(C.D, ct2, o2);
#pragma unroll
    for (int t = 0; t < n; ++t) I[a1 + n * t] = o[t] + o2[t];
    mat_line<T, n, true>(C.S, ct1, o);
#pragma unroll
    for (int t = 0; t < n; ++t) I[n2 + a1 + n * t] = o[t];
    mat_line<T, n, true>(C.S, cd, o);
#pragma unroll
    for (int t = 0; t < n; ++t) I[2 * n2 + a1 + n * t] = o[t];
  }
  __syncthreads();
  // ---- F3: per (cell, face, node i2): transposed pass along t1: FL = S^T I0 + D^T I1, GL = S^T I2
  // (face-node coefficients of the layer value and of the normal derivative; over AS)
  for (int it = tid; it < cpb * 6 * n; it += nt) {
    const int c = it / (6 * n), r = it - c * 6 * n, f = r / n, i2 = r % n;
    T *cc = sm + c * PL::per_cell;
    const T *I = cc + PL::LAY + f * 3 * n2;
    T v0[n], v1[n], v2[n], o[n], o2[n];
#pragma unroll
    for (int a = 0; a < n; ++a) { v0[a] = I[a + n * i2]; v1[a] = I[n2 + a + n * i2]; v2[a] = I[2 * n2 + a + n * i2]; }
    mat_line<T, n, true>(C.S, v0, o);
    mat_line<T, n, true>(C.D, v1, o2);
    T *FL = cc + PL::AS + f * 2 * n2;
#pragma unroll
    for (int t = 0; t < n; ++t) FL[t + n * i2] = o[t] + o2[t];
    mat_line<T, n, true>(C.S, v2, o);
#pragma unroll
    for (int t = 0; t < n; ++t) FL[n2 + t + n * i2] = o[t];
  }
  __syncthreads();
  // ---- P5: x-lines at (y, z) = (lr, lq): D^T V0 + S^T V1, plus the six faces' coefficients
  if (line) {
    T v0[n], v1[n], o[n], o2[n];
#pragma unroll
    for (int t = 0; t < n; ++t) { v0[t] = cs[PL::X0 + n * l + t]; v1[t] = cs[PL::X1 + n * l + t]; }
    mat_line<T, n, true>(C.D, v0, o);
    mat_line<T, n, true>(C.S, v1, o2);
    const T *FL = cs + PL::AS;
#pragma unroll
    for (int x = 0; x < n; ++x) {
      T s = o[x] + o2[x];
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const T *Fx = FL + (0 + sd) * 2 * n2, *Fy = FL + (2 + sd) * 2 * n2, *Fz = FL + (4 + sd) * 2 * n2;
        const int e = sd ? n - 1 : 0;
        // x-faces: node (y, z) = l; y-faces: node (x, z) = x + n lq; z-faces: node (x, y) = x + n lr
        s += C.E[sd][x] * Fx[n2 + l] + (x == e ? Fx[l] : T(0));
        s += C.E[sd][lr] * Fy[n2 + x + n * lq] + (lr == e ? Fy[x + n * lq] : T(0));
        s += C.E[sd][lq] * Fz[n2 + x + n * lr] + (lq == e ? Fz[x + n * lr] : T(0));
      }
      const size_t i = (size_t)(c0 + cl) * n3 + n * l + x;
      if (epi.mode == LAP_PLAIN) {
        y[i] = s;
      } else if (epi.mode == LAP_RESIDUAL) {
        y[i] = epi.b[i] - s;
      } else {
        const T dn = (epi.first ? T(0) : epi.c1 * epi.d[i]) + epi.c2 * epi.dinv[i] * (epi.b[i] - s);
        epi.d[i] = dn;
        epi.xout[i] = p[i] + dn;
      }
    }
  }
}

static int curved_cpb(int nx, int n) {
  int c = 1;
  while (c * 2 <= 4 && (c * 2) * n * n <= 256 && nx % (c * 2) == 0) c *= 2;
  return c;
}

template <typename T, int K>
static cudaError_t launch_curved_k(const MeshView<T> &m, const T *p, T *y, const LapEpi<T> &epi, cudaStream_t s) {
  constexpr int n = K + 1;
  const int cpb = curved_cpb(m.nx, n);
  const size_t sm = sizeof(T) * (size_t)cpb * CurvPlan<n>::per_cell + sizeof(int) * cpb * 6;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(curved_laplace_kernel<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         160 * 1024);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(curved_laplace_kernel<T, K>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int threads = ((cpb * n * n + 31) / 32) * 32;
  note_launch();
  note_dofs(m.np);
  curved_laplace_kernel<T, K><<<m.nc / cpb, threads, sm, s>>>(m, p, y, cpb, epi);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_curved_laplace(const MeshView<T> &m, const T *p, T *y, const LapEpi<T> &epi, cudaStream_t s) {
  switch (m.n1) {
    case 2: return launch_curved_k<T, 1>(m, p, y, epi, s);
    case 3: return launch_curved_k<T, 2>(m, p, y, epi, s);
    case 4: return launch_curved_k<T, 3>(m, p, y, epi, s);
    case 5: return launch_curved_k<T, 4>(m, p, y, epi, s);
    case 6: return launch_curved_k<T, 5>(m, p, y, epi, s);
  }
  return cudaErrorInvalidValue;
}

template cudaError_t launch_curved_laplace<double>(const MeshView<double> &, const double *, double *,
                                                   const LapEpi<double> &, cudaStream_t);
template cudaError_t launch_curved_laplace<float>(const MeshView<float> &, const float *, float *,
                                                  const LapEpi<float> &, cudaStream_t);

}  // namespace dgw
