// SIPG Laplacian on the channel of boxes, specialised by degree (Sec. 4.2 eq. ipflux, Sec. 4.4
// sum factorisation).
//
// On an axis-aligned box cell with exact Gauss integration, the cell and face integrals of the
// SIPG form factorise per direction: with the 1-D reference mass matrix M,
//   y_c = sum_d (L_d (x)_d M (x) M) u_c + sum_{d,s} (N_{d,s} (x)_d M (x) M) u_{nb(d,s)},
// where L_d (n x n) holds the stiffness along d plus the own-side face terms of both faces
// normal to d, and N_{d,s} is the rank-2 coupling to the neighbour across face s, which only
// needs the neighbour's trace value and reference normal derivative on the shared face. L_d and
// the coupling vectors depend only on the cell row j (graded spacing, penalty), so they are
// tabulated per row on the host (box_rowops) and staged in shared memory.
//
// Evaluation: y = M_z [ M_y (L_x u + nbr_x) + L_y (M_x u) + nbr_y' ] + L_z (M_x M_y u) + nbr_z'',
// three line passes (one thread owns a whole 1-D line in registers), with the y-face traces
// transformed by M_x and the z-face traces by M_x M_y. A CTA holds cpb consecutive cells along x.
#include "sumfac.cuh"

namespace dgw {

// Per-row operator layout: Lx, Ly, Lz (n*n each), then for d in {x,y,z}, s in {0,1}: c1[n], c2[n].
__host__ __device__ constexpr int rowops_size(int n) { return 3 * n * n + 12 * n; }

// FP32: up to 3 CTAs of <= 256 threads per SM for k <= 4 (register budget ~85/thread), 2 for k = 5;
// FP64 is FP64-pipe bound and keeps the default budget.
template <typename T, int K>
struct BoxOcc { static constexpr int min_blocks = 1; };
template <int K>
struct BoxOcc<float, K> { static constexpr int min_blocks = K <= 4 ? 3 : 2; };

template <typename T, int K>
__global__ void __launch_bounds__(256, (BoxOcc<T, K>::min_blocks)) laplace_box_kernel(MeshView<T> m, const T *__restrict__ p,
                                                                                T *__restrict__ y, int cpb) {
  constexpr int n = K + 1, n2 = n * n, n3 = n2 * n;
  constexpr int ROW = rowops_size(n);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Ms = reinterpret_cast<T *>(smem_raw);   // n2
  T *Dd = Ms + n2;                             // 2n: l_j'(0), l_j'(1)
  T *R = Dd + 2 * n;                           // ROW
  T *U = R + ROW;                              // cpb n3 (input, then output)
  T *A = U + cpb * n3;                         // cpb n3 (T1 -> W)
  T *B = A + cpb * n3;                         // cpb n3 (T2 -> T3)
  T *TR = B + cpb * n3;                        // cpb * 6 faces * 2 (val, der) * n2
  T *TY = TR + cpb * 24 * n2;                  // cpb * 2 faces * 2 * n2 : y-face traces after M_x
  T *TZ = TY + cpb * 8 * n2;                   // cpb * 2 * 2 * n2 : z-face traces after M_x
  const int tid = threadIdx.x, nt = blockDim.x;
  const int c0 = blockIdx.x * cpb;
  const int i0 = c0 % m.nx, j = (c0 / m.nx) % m.ny, kz = c0 / (m.nx * m.ny);
  const Basis<T> *Bg = m.basis;
  for (int t = tid; t < n2; t += nt) Ms[t] = Bg->mass[t];
  for (int t = tid; t < n; t += nt) { Dd[t] = Bg->dend[0][t]; Dd[n + t] = Bg->dend[1][t]; }
  const T *Rg = m.rowops + (size_t)j * ROW;
  for (int t = tid; t < ROW; t += nt) R[t] = Rg[t];
  const T *pc = p + (size_t)c0 * n3;
  for (int t = tid; t < cpb * n3; t += nt) U[t] = pc[t];
  __syncthreads();   // Dd, Ms and R are read by every thread below
  // neighbour traces: value and reference normal derivative on the shared face
  for (int t = tid; t < cpb * 6 * n2; t += nt) {
    const int cl = t / (6 * n2), f = (t / n2) % 6, node = t % n2;
    const int d = f >> 1, side = f & 1;
    int ii = i0 + cl, jj = j, kk = kz;
    const int sg = side ? 1 : -1;
    bool wall = false;
    if (d == 0) ii = (ii + sg + m.nx) % m.nx;
    else if (d == 2) kk = (kk + sg + m.nz) % m.nz;
    else { jj += sg; wall = jj < 0 || jj >= m.ny; }
    T val = T(0), der = T(0);
    if (!wall) {
      const T *pn = p + ((size_t)ii + (size_t)m.nx * (jj + (size_t)m.ny * kk)) * n3;
      const int t1 = node % n, t2 = node / n;
      // neighbour endpoint on the shared face: side 0 -> its xi_d = 1, side 1 -> its xi_d = 0
      const int ep = side ? 0 : 1;
      const T *dv = Dd + ep * n;
      int stride, base;
      if (d == 0) { stride = 1; base = n * (t1 + n * t2); }
      else if (d == 1) { stride = n; base = t1 + n2 * t2; }
      else { stride = n2; base = t1 + n * t2; }
      const int lay = ep ? n - 1 : 0;
      val = pn[base + lay * stride];
#pragma unroll
      for (int b = 0; b < n; ++b) der += dv[b] * pn[base + b * stride];
    }
    TR[((cl * 6 + f) * 2 + 0) * n2 + node] = val;
    TR[((cl * 6 + f) * 2 + 1) * n2 + node] = der;
  }
  __syncthreads();
  const T *Lx = R, *Ly = R + n2, *Lz = R + 2 * n2;
  auto c1 = [&](int d, int s) -> const T * { return R + 3 * n2 + (d * 2 + s) * 2 * n; };
  auto c2 = [&](int d, int s) -> const T * { return R + 3 * n2 + (d * 2 + s) * 2 * n + n; };
  // ---- phase A: x-lines (T1 = Lx u + nbr_x, T2 = M_x u); y-traces <- M_x; z-traces <- M_x
  {
    const int nlines = cpb * n2, nty = cpb * 4 * n, total = nlines + 2 * nty;
    for (int t = tid; t < total; t += nt) {
      if (t < nlines) {
        const int cl = t / n2, l = t % n2;
        const int base = cl * n3 + n * l;
        T u[n], o1[n], o2[n];
#pragma unroll
        for (int b = 0; b < n; ++b) u[b] = U[base + b];
        const T v0 = TR[((cl * 6 + 0) * 2 + 0) * n2 + l], d0 = TR[((cl * 6 + 0) * 2 + 1) * n2 + l];
        const T v1 = TR[((cl * 6 + 1) * 2 + 0) * n2 + l], d1 = TR[((cl * 6 + 1) * 2 + 1) * n2 + l];
        const T *a0 = c1(0, 0), *b0 = c2(0, 0), *a1 = c1(0, 1), *b1 = c2(0, 1);
#pragma unroll
        for (int a = 0; a < n; ++a) {
          T s1 = a0[a] * v0 + b0[a] * d0 + a1[a] * v1 + b1[a] * d1, s2 = T(0);
#pragma unroll
          for (int b = 0; b < n; ++b) {
            s1 += Lx[a * n + b] * u[b];
            s2 += Ms[a * n + b] * u[b];
          }
          o1[a] = s1;
          o2[a] = s2;
        }
#pragma unroll
        for (int a = 0; a < n; ++a) { A[base + a] = o1[a]; B[base + a] = o2[a]; }
      } else {
        // trace transform along x (t1 axis of y- and z-faces): item = (cl, face, arr, t2)
        const int r = t - nlines;
        const bool isz = r >= nty;
        const int q = isz ? r - nty : r;
        const int cl = q / (4 * n), fa = (q / n) % 4, t2 = q % n;   // fa = 2*face + (val|der)
        const int fl = fa >> 1, arr = fa & 1;
        const int f = (isz ? 4 : 2) + fl;
        const T *src = TR + ((cl * 6 + f) * 2 + arr) * n2 + n * t2;
        T *dst = (isz ? TZ : TY) + ((cl * 2 + fl) * 2 + arr) * n2 + n * t2;
        T v[n];
#pragma unroll
        for (int b = 0; b < n; ++b) v[b] = src[b];
#pragma unroll
        for (int a = 0; a < n; ++a) {
          T s = T(0);
#pragma unroll
          for (int b = 0; b < n; ++b) s += Ms[a * n + b] * v[b];
          dst[a] = s;
        }
      }
    }
  }
  __syncthreads();
  // ---- phase B: y-lines (W = M_y T1 + Ly T2 + nbr_y', T3 = M_y T2); z-traces <- M_y (into TR z slots)
  {
    const int nlines = cpb * n2, ntz = cpb * 4 * n, total = nlines + ntz;
    for (int t = tid; t < total; t += nt) {
      if (t < nlines) {
        const int cl = t / n2, x = t % n, z = (t / n) % n;
        const int base = cl * n3 + x + n2 * z;
        T a1[n], a2[n], w[n], t3[n];
#pragma unroll
        for (int c = 0; c < n; ++c) { a1[c] = A[base + n * c]; a2[c] = B[base + n * c]; }
        const int fi = x + n * z;
        const T v0 = TY[((cl * 2 + 0) * 2 + 0) * n2 + fi], d0 = TY[((cl * 2 + 0) * 2 + 1) * n2 + fi];
        const T v1 = TY[((cl * 2 + 1) * 2 + 0) * n2 + fi], d1 = TY[((cl * 2 + 1) * 2 + 1) * n2 + fi];
        const T *e0 = c1(1, 0), *g0 = c2(1, 0), *e1 = c1(1, 1), *g1 = c2(1, 1);
#pragma unroll
        for (int b = 0; b < n; ++b) {
          T s = e0[b] * v0 + g0[b] * d0 + e1[b] * v1 + g1[b] * d1, s3 = T(0);
#pragma unroll
          for (int c = 0; c < n; ++c) {
            s += Ms[b * n + c] * a1[c] + Ly[b * n + c] * a2[c];
            s3 += Ms[b * n + c] * a2[c];
          }
          w[b] = s;
          t3[b] = s3;
        }
#pragma unroll
        for (int b = 0; b < n; ++b) { A[base + n * b] = w[b]; B[base + n * b] = t3[b]; }
      } else {
        // z-face traces (indexed x + n*y) after M_x: apply M_y along t2 = y; item = (cl, fl, arr, x)
        const int q = t - nlines;
        const int cl = q / (4 * n), pr = (q / n) % 4, x = q % n;
        const int fl = pr >> 1, arr = pr & 1;
        const T *src = TZ + ((cl * 2 + fl) * 2 + arr) * n2 + x;
        T *dst = TR + ((cl * 6 + 4 + fl) * 2 + arr) * n2 + x;
        T v[n];
#pragma unroll
        for (int b = 0; b < n; ++b) v[b] = src[n * b];
#pragma unroll
        for (int a = 0; a < n; ++a) {
          T s = T(0);
#pragma unroll
          for (int b = 0; b < n; ++b) s += Ms[a * n + b] * v[b];
          dst[n * a] = s;
        }
      }
    }
  }
  __syncthreads();
  // ---- phase C: z-lines (y = M_z W + Lz T3 + nbr_z'')
  for (int t = tid; t < cpb * n2; t += nt) {
    const int cl = t / n2, l = t % n2;   // l = x + n*y
    const int base = cl * n3 + l;
    T a1[n], a2[n];
#pragma unroll
    for (int e = 0; e < n; ++e) { a1[e] = A[base + n2 * e]; a2[e] = B[base + n2 * e]; }
    const T v0 = TR[((cl * 6 + 4) * 2 + 0) * n2 + l], d0 = TR[((cl * 6 + 4) * 2 + 1) * n2 + l];
    const T v1 = TR[((cl * 6 + 5) * 2 + 0) * n2 + l], d1 = TR[((cl * 6 + 5) * 2 + 1) * n2 + l];
    const T *e0 = c1(2, 0), *g0 = c2(2, 0), *e1 = c1(2, 1), *g1 = c2(2, 1);
#pragma unroll
    for (int c = 0; c < n; ++c) {
      T s = e0[c] * v0 + g0[c] * d0 + e1[c] * v1 + g1[c] * d1;
#pragma unroll
      for (int e = 0; e < n; ++e) s += Ms[c * n + e] * a1[e] + Lz[c * n + e] * a2[e];
      U[base + n2 * c] = s;
    }
  }
  __syncthreads();
  T *yc = y + (size_t)c0 * n3;
  for (int t = tid; t < cpb * n3; t += nt) yc[t] = U[t];
}

template <typename T>
static size_t box_smem(int n, int cpb) {
  const int n2 = n * n, n3 = n2 * n;
  return sizeof(T) * ((size_t)n2 + 2 * n + rowops_size(n) + 3 * (size_t)cpb * n3 + (size_t)cpb * (24 + 8 + 8) * n2);
}

// cells per CTA: the largest power of two dividing nx with cpb*(k+1)^2 <= 256 and cpb <= 8
static int box_cpb(int nx, int n) {
  int c = 1;
  while (c * 2 <= 8 && (c * 2) * n * n <= 256 && nx % (c * 2) == 0) c *= 2;
  return c;
}

template <typename T, int K>
static cudaError_t launch_box_k(const MeshView<T> &m, const T *p, T *y, cudaStream_t s) {
  constexpr int n = K + 1;
  const int cpb = box_cpb(m.nx, n);
  const size_t sm = box_smem<T>(n, cpb);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(laplace_box_kernel<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e == cudaSuccess)   // the whole unified L1/shared array as shared memory: more CTAs per SM
      e = cudaFuncSetAttribute(laplace_box_kernel<T, K>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int threads = ((cpb * n * n + 31) / 32) * 32;
  note_launch();
  note_dofs(m.np);
  laplace_box_kernel<T, K><<<m.nc / cpb, threads, sm, s>>>(m, p, y, cpb);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_laplace(const MeshView<T> &m, const T *p, T *y, cudaStream_t s) {
  if (m.geo == GEO_CURVED) return launch_vector_op<T>(OP_LAP, m, p, y, s);   // per-point metrics
  switch (m.n1) {
    case 2: return launch_box_k<T, 1>(m, p, y, s);
    case 3: return launch_box_k<T, 2>(m, p, y, s);
    case 4: return launch_box_k<T, 3>(m, p, y, s);
    case 5: return launch_box_k<T, 4>(m, p, y, s);
    case 6: return launch_box_k<T, 5>(m, p, y, s);
  }
  return cudaErrorInvalidValue;
}

template cudaError_t launch_laplace<double>(const MeshView<double> &, const double *, double *, cudaStream_t);
template cudaError_t launch_laplace<float>(const MeshView<float> &, const float *, float *, cudaStream_t);

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
