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
#include <cstdint>
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

// Register budget through the CTAs per SM the kernel is compiled for: FP32 56 registers a thread
// (5 CTAs of 224 threads for k = 4), FP64 is FP64-pipe bound and keeps the default budget,
// double-float (two registers per value, about fifteen instructions per multiply-add) two CTAs.
template <typename T, int NT>
struct BoxOcc { static constexpr int min_blocks = 1; };
template <int NT>
struct BoxOcc<float, NT> {
  static constexpr int v = 65536 / (NT * 56);
  static constexpr int min_blocks = v < 1 ? 1 : (v > 8 ? 8 : v);
};
template <int NT>
struct BoxOcc<df64, NT> { static constexpr int min_blocks = 2; };

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

// Shared-memory bank layout. Thread t owns line t / CPB of cell t % CPB (the cells of a warp
// interleave), and every per-cell array has a padded cell stride. bank_cost counts the wavefronts
// (the largest number of lanes on one 4-byte bank, summed over the warps) of the accesses
// a(t) = stride * cell + f(line) of the three line passes: x-lines n l, y-lines (l mod n) + n^2 (l / n),
// z-lines l (and the face-node index l of the traces); the stride with the fewest wavefronts in
// [base, base + 32) wins. For k = 4 and 8 cells the stride 148 (= 20 mod 32) makes all three passes
// conflict-free.
constexpr int bank_cost(int stride, int n, int cpb, int pattern, bool cell_major = false, int lim = 1 << 30) {
  int total = 0;
  const int lines = cpb * n * n;
  for (int w = 0; w * 32 < lines; ++w) {
    int cnt[32] = {};
    int mx = 0;
    for (int i = 0; i < 32; ++i) {
      const int t = w * 32 + i;
      if (t >= lines) break;
      const int cl = cell_major ? t / (n * n) : t % cpb, l = cell_major ? t % (n * n) : t / cpb;
      if (l >= lim) continue;
      const int f = pattern == 0 ? n * l : (pattern == 1 ? (l % n) + n * n * (l / n) : l);
      const int b = (stride * cl + f) % 32;
      if (++cnt[b] > mx) mx = cnt[b];
    }
    total += mx;
  }
  return total;
}
// kind 0: U, A, B (the three line passes); 1: the six-face trace array (written cell-major, 12 stores
// a thread; read by the x- and z-passes, 4 loads each; M_x and M_y transform items of the first 4n
// lines); 2: the y- and z-face arrays after M_x (transform writes, 4 loads of the y-pass)
constexpr int stride_cost(int st, int n, int cpb, int kind) {
  if (kind == 0) return bank_cost(st, n, cpb, 0) + bank_cost(st, n, cpb, 1) + bank_cost(st, n, cpb, 2);
  if (kind == 1)
    return 12 * bank_cost(st, n, cpb, 2, true) + 8 * bank_cost(st, n, cpb, 2) + 2 * n * bank_cost(st, n, cpb, 0, false, 4 * n) +
           n * bank_cost(st, n, cpb, 1, false, 4 * n);
  return 2 * n * bank_cost(st, n, cpb, 0, false, 4 * n) + 4 * bank_cost(st, n, cpb, 2) + n * bank_cost(st, n, cpb, 1, false, 4 * n);
}
constexpr int best_stride(int base, int n, int cpb, int kind) {
  int best = base, cost = 1 << 30;
  for (int pad = 0; pad < 32; ++pad) {
    const int c = stride_cost(base + pad, n, cpb, kind);
    if (c < cost) { cost = c; best = base + pad; }
  }
  return best;
}

// Launch shape of a CTA of CPB cells (a row segment along x): one thread per line of every cell.
template <int K, int CPB>
struct BoxShape {
  static constexpr int n = K + 1, n2 = n * n, n3 = n2 * n;
  static constexpr int lines = CPB * n2;
  static constexpr int threads = ((lines + 31) / 32) * 32;
  static constexpr int S = best_stride(n3, n, CPB, 0);        // cell stride of U, A, B
  static constexpr int TS = best_stride(12 * n2, n, CPB, 1);  // six faces x (value, derivative)
  static constexpr int YS = best_stride(4 * n2, n, CPB, 2);   // two faces x (value, derivative)
  // shared memory in compute-type words: row scalars (padded to 32), U, A, B, traces of the six
  // faces, y- and z-face traces after M_x
  static constexpr int rs = 32;
  static constexpr int words = rs + 3 * CPB * S + CPB * TS + 2 * CPB * YS;
};

// 16-byte vector of the storage type
template <typename T>
struct Vec16;
template <>
struct Vec16<float> { using type = float4; static constexpr int w = 4; };
template <>
struct Vec16<double> { using type = double2; static constexpr int w = 2; };

template <typename V>
__device__ __forceinline__ V vload(const void *p) { return *reinterpret_cast<const V *>(p); }

// y_j = f(j) over the CTA's CPB n^3 values: 16-byte vectors when the element type allows it (T == R)
// and every pointer of the call is 16-byte aligned, else one value per thread and step.
template <typename T, int N, int NT, typename F>
__device__ __forceinline__ void span_for(bool vec, F f) {
  constexpr int W = Vec16<T>::w;
  if (vec) {
#pragma unroll 4
    for (int v = threadIdx.x; v < N / W; v += NT) f(v * W, std::integral_constant<int, W>{});
  } else {
#pragma unroll 4
    for (int t = threadIdx.x; t < N; t += NT) f(t, std::integral_constant<int, 1>{});
  }
}

__device__ __forceinline__ bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// T: storage type of p and y; R: compute type (T itself, or df64 for FP64-accurate arithmetic on the
// FP32 units with double vectors; that variant supports the plain epilogue only). CPB cells per CTA.
template <typename T, typename R, int K, int CPB>
__global__ void __launch_bounds__(BoxShape<K, CPB>::threads, (BoxOcc<R, BoxShape<K, CPB>::threads>::min_blocks))
    laplace_box_kernel(MeshView<T> m, const T *__restrict__ p, T *__restrict__ y, LapEpi<T> epi) {
  using S = BoxShape<K, CPB>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, NT = S::threads, NV = CPB * n3;
  constexpr int CS = S::S, TS = S::TS, YS = S::YS;
  constexpr bool SAME = std::is_same<T, R>::value;
  constexpr bool VECOK = SAME && (NV * sizeof(T)) % 16 == 0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *Rs = reinterpret_cast<R *>(smem_raw);     // kRowScal
  R *U = Rs + S::rs;                            // CPB cells of stride CS (input, then output)
  R *A = U + CPB * CS;                          // (T1 -> W)
  R *B = A + CPB * CS;                          // (T2 -> T3)
  R *TR = B + CPB * CS;                         // CPB x [6 faces x 2 (val, der) x n2], stride TS
  R *TY = TR + CPB * TS;                        // CPB x [2 faces x 2 x n2], stride YS: y-face traces after M_x
  R *TZ = TY + CPB * YS;                        // the same for the z-faces
  const BoxConst<R> &C = box_const<R>(K);
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * CPB;
  if (blockIdx.y > 0) {   // column blockIdx.y of a block of vectors (the diagonal dinv is shared)
    const size_t co = (size_t)blockIdx.y * m.np;
    p += co;
    if (y) y += co;
    if (epi.b) epi.b += co;
    if (epi.d) epi.d += co;
    if (epi.xout) epi.xout += co;
  }
  const int nx = m.nx, ny = m.ny, nz = m.nz;
  const int rowid = c0 / nx, kz = rowid / ny;
  const int i0 = c0 - rowid * nx, j = rowid - kz * ny;
  const T *Rg = m.rowops + (size_t)j * kRowScal;
  if (tid < kRowScal) Rs[tid] = r_load<R>(Rg[tid]);
  const size_t o = (size_t)c0 * n3;
  const T *pc = p + o;
  // value t of the CTA's cells -> its padded slot
  auto slot = [](int t) { const int c = t / n3; return c * CS + (t - c * n3); };
  // one value per thread and step: consecutive lanes store consecutive slots (16-byte loads would
  // store four slots 4 apart per lane, a 4-way bank conflict in the padded layout)
#pragma unroll 4
  for (int t = tid; t < NV; t += NT) U[slot(t)] = r_load<R>(pc[t]);
  // Every thread owns line l of cell cl in all three passes (x-, y- then z-lines; l indexes the
  // face nodes of the same two tangential axes), so the index arithmetic is done once here.
  const bool line = tid < S::lines;
  const int cl = line ? tid % CPB : 0, l = line ? tid / CPB : 0;
  const int lq = l / n, lr = l - lq * n;   // l = lr + n * lq
  __syncthreads();
  // neighbour traces at face node l of the six faces: value and reference normal derivative. This
  // phase maps threads to lines cell by cell (tc = tid / n^2), so a warp's neighbour loads fall on
  // one or two neighbour cells and the in-segment test for the x-faces is uniform in most warps.
  if (line) {
    const int cl = tid / n2, l = tid - cl * n2, lq = l / n, lr = l - lq * n;
    const int ci = i0 + cl;
    R *tr = TR + cl * TS + l;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1, side = f & 1;
      const int sg = side ? 1 : -1;
      // neighbour endpoint on the shared face: side 0 -> its xi_d = 1, side 1 -> its xi_d = 0
      const int stride = d == 0 ? 1 : (d == 1 ? n : n2);
      const int base = d == 0 ? n * l : (d == 1 ? lr + n2 * lq : l);
      R v[n];
      bool has = true;
      if (d == 0 && cl + sg >= 0 && cl + sg < CPB) {   // x-neighbour inside the row segment
        const R *pn = U + (cl + sg) * CS + base;
#pragma unroll
        for (int b = 0; b < n; ++b) v[b] = pn[b * stride];
      } else {
        int ii = ci, jj = j, kk = kz;   // periodic in x and z
        if (d == 0) {
          ii = ci + sg;
          ii += ii < 0 ? nx : 0;
          ii -= ii >= nx ? nx : 0;
        } else if (d == 1) {
          jj = j + sg;
        } else {
          kk = kz + sg;
          kk += kk < 0 ? nz : 0;
          kk -= kk >= nz ? nz : 0;
        }
        has = jj >= 0 && jj < ny;
        const T *pn = p + (size_t)(ii + nx * (jj + ny * kk)) * n3 + base;
#pragma unroll
        for (int b = 0; b < n; ++b) v[b] = has ? r_load<R>(pn[b * stride]) : r_zero<R>();
      }
      R der = r_zero<R>();
#pragma unroll
      for (int b = 0; b < n; ++b) der = r_fma(side ? C.D[0][b] : C.D[1][b], v[b], der);
      tr[(f * 2 + 0) * n2] = has ? (side ? v[0] : v[n - 1]) : r_zero<R>();
      tr[(f * 2 + 1) * n2] = der;
    }
  }
  __syncthreads();
  // ---- phase A: x-lines (T1 = Lx u + nbr_x, T2 = M_x u); y- and z-traces <- M_x (items
  // it = l, l + n^2, ... < 4n: face (it / n) >> 1, array (it / n) & 1, t2 = it % n)
  if (line) {
    const int base = cl * CS + n * l;
    const R *tr = TR + cl * TS + l;
    R u[n], o1[n], o2[n];
#pragma unroll
    for (int b = 0; b < n; ++b) u[b] = U[base + b];
    line_op<R, K>(u, Rs, tr[0], tr[n2], tr[2 * n2], tr[3 * n2], o1);
    mass_line<R, K>(u, o2);
#pragma unroll
    for (int a = 0; a < n; ++a) { A[base + a] = o1[a]; B[base + a] = o2[a]; }
    for (int it = l; it < 4 * n; it += n2) {   // one item per thread for k >= 3
      const int iq = it / n, ir = it - iq * n;
      const int fl = iq >> 1, arr = iq & 1;
#pragma unroll
      for (int isz = 0; isz < 2; ++isz) {
        const R *src = TR + cl * TS + (((isz ? 4 : 2) + fl) * 2 + arr) * n2 + n * ir;
        R *dst = (isz ? TZ : TY) + cl * YS + (fl * 2 + arr) * n2 + n * ir;
        R v[n], ov[n];
#pragma unroll
        for (int b = 0; b < n; ++b) v[b] = src[b];
        mass_line<R, K>(v, ov);
#pragma unroll
        for (int a = 0; a < n; ++a) dst[a] = ov[a];
      }
    }
  }
  __syncthreads();
  // ---- phase B: y-lines at (x, z) = (lr, lq): W = M_y T1 + Ly T2 + nbr_y', T3 = M_y T2; z-face
  // traces (indexed x + n*y) <- M_y (items it as in phase A, x = it % n)
  if (line) {
    const int base = cl * CS + lr + n2 * lq;
    const R *ty = TY + cl * YS + l;
    R a1[n], a2[n], w[n], t3[n], ly[n];
#pragma unroll
    for (int c = 0; c < n; ++c) { a1[c] = A[base + n * c]; a2[c] = B[base + n * c]; }
    line_op<R, K>(a2, Rs + 8, ty[0], ty[n2], ty[2 * n2], ty[3 * n2], ly);
    mass_line<R, K>(a1, w);
    mass_line<R, K>(a2, t3);
#pragma unroll
    for (int b = 0; b < n; ++b) { A[base + n * b] = w[b] + ly[b]; B[base + n * b] = t3[b]; }
    for (int it = l; it < 4 * n; it += n2) {
      const int iq = it / n, ir = it - iq * n;
      const int fl = iq >> 1, arr = iq & 1;
      const R *src = TZ + cl * YS + (fl * 2 + arr) * n2 + ir;
      R *dst = TR + cl * TS + ((4 + fl) * 2 + arr) * n2 + ir;
      R v[n], ov[n];
#pragma unroll
      for (int b = 0; b < n; ++b) v[b] = src[n * b];
      mass_line<R, K>(v, ov);
#pragma unroll
      for (int a = 0; a < n; ++a) dst[n * a] = ov[a];
    }
  }
  __syncthreads();
  // ---- phase C: z-lines at l = x + n*y (y = M_z W + Lz T3 + nbr_z'')
  if (line) {
    const int base = cl * CS + l;
    const R *tz = TR + cl * TS + 8 * n2 + l;
    R a1[n], a2[n], w[n], lz[n];
#pragma unroll
    for (int e = 0; e < n; ++e) { a1[e] = A[base + n2 * e]; a2[e] = B[base + n2 * e]; }
    line_op<R, K>(a2, Rs + 16, tz[0], tz[n2], tz[2 * n2], tz[3 * n2], lz);
    mass_line<R, K>(a1, w);
#pragma unroll
    for (int c = 0; c < n; ++c) U[base + n2 * c] = w[c] + lz[c];
  }
  __syncthreads();
  if (epi.mode == LAP_PLAIN) {
    T *yo = y + o;
    if constexpr (VECOK) {
      using V = typename Vec16<T>::type;
      span_for<T, NV, NT>(aligned16(yo), [&](int t, auto w) {
        if constexpr (decltype(w)::value > 1) {
          T v[Vec16<T>::w];
#pragma unroll
          for (int q = 0; q < Vec16<T>::w; ++q) v[q] = U[slot(t + q)];
          *reinterpret_cast<V *>(yo + t) = *reinterpret_cast<const V *>(v);
        } else {
          yo[t] = U[slot(t)];
        }
      });
    } else {
      for (int t = tid; t < NV; t += NT) yo[t] = r_store<T>(U[slot(t)]);
    }
  } else if constexpr (SAME) {
    constexpr int W = Vec16<T>::w;
    if (epi.mode == LAP_RESIDUAL) {
      T *yo = y + o;
      const T *bo = epi.b + o;
      span_for<T, NV, NT>(VECOK && aligned16(yo) && aligned16(bo), [&](int t, auto w) {
        if constexpr (decltype(w)::value > 1) {
          using V = typename Vec16<T>::type;
          T bv[W], r[W];
          *reinterpret_cast<V *>(bv) = vload<V>(bo + t);
#pragma unroll
          for (int q = 0; q < W; ++q) r[q] = bv[q] - U[slot(t + q)];
          *reinterpret_cast<V *>(yo + t) = *reinterpret_cast<const V *>(r);
        } else {
          yo[t] = bo[t] - U[slot(t)];
        }
      });
    } else {
      const T *bo = epi.b + o, *dio = epi.dinv + o, *po = p + o;
      T *dd = epi.d + o, *xo = epi.xout + o;
      const T c1 = epi.first ? T(0) : epi.c1, c2 = epi.c2;
      const bool first = epi.first != 0;
      const bool vec = VECOK && aligned16(bo) && aligned16(dio) && aligned16(po) && aligned16(dd) && aligned16(xo);
      span_for<T, NV, NT>(vec, [&](int t, auto w) {
        if constexpr (decltype(w)::value > 1) {
          using V = typename Vec16<T>::type;
          T bv[W], di[W], pv[W], dv[W], dn[W], xv[W];
          *reinterpret_cast<V *>(bv) = vload<V>(bo + t);
          *reinterpret_cast<V *>(di) = vload<V>(dio + t);
          *reinterpret_cast<V *>(pv) = vload<V>(po + t);
          if (!first) *reinterpret_cast<V *>(dv) = vload<V>(dd + t);
#pragma unroll
          for (int q = 0; q < W; ++q) {
            dn[q] = (first ? T(0) : c1 * dv[q]) + c2 * di[q] * (bv[q] - U[slot(t + q)]);
            xv[q] = pv[q] + dn[q];
          }
          *reinterpret_cast<V *>(dd + t) = *reinterpret_cast<const V *>(dn);
          *reinterpret_cast<V *>(xo + t) = *reinterpret_cast<const V *>(xv);
        } else {
          const T dn = (first ? T(0) : c1 * dd[t]) + c2 * dio[t] * (bo[t] - U[slot(t)]);
          dd[t] = dn;
          xo[t] = po[t] + dn;
        }
      });
    }
  }
}

template <typename T, int K, int CPB>
static size_t box_smem() {
  return sizeof(T) * (size_t)BoxShape<K, CPB>::words;
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

template <typename T, typename R, int K, int CPB>
static cudaError_t launch_box_kc(const MeshView<T> &m, const T *p, T *y, const LapEpi<T> &epi, cudaStream_t s) {
  using S = BoxShape<K, CPB>;
  const size_t sm = box_smem<R, K, CPB>();
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    // the whole unified L1/shared array as shared memory: more CTAs per SM
    attr_err = cudaFuncSetAttribute(laplace_box_kernel<T, R, K, CPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    160 * 1024);
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(laplace_box_kernel<T, R, K, CPB>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  });
  if (attr_err != cudaSuccess) return attr_err;
  const int ncols = epi.ncols > 1 ? epi.ncols : 1;
  note_launch();
  note_dofs(m.np * ncols);
  laplace_box_kernel<T, R, K, CPB><<<dim3(m.nc / CPB, ncols), S::threads, sm, s>>>(m, p, y, epi);
  return cudaGetLastError();
}

template <typename T, typename R, int K>
static cudaError_t launch_box_k(const MeshView<T> &m, const T *p, T *y, const LapEpi<T> &epi, cudaStream_t s) {
  constexpr int n = K + 1;
  switch (box_cpb(m.nx, n)) {
    case 8:
      if constexpr (8 * n * n <= 256) return launch_box_kc<T, R, K, 8>(m, p, y, epi, s);
      break;
    case 4: return launch_box_kc<T, R, K, 4>(m, p, y, epi, s);
    case 2: return launch_box_kc<T, R, K, 2>(m, p, y, epi, s);
    case 1: return launch_box_kc<T, R, K, 1>(m, p, y, epi, s);
  }
  return cudaErrorInvalidValue;
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
