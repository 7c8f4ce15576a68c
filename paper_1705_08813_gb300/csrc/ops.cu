// Matrix-free DG operators with one CTA per cell: the volume integral of the cell and the integrals
// over its six faces for its own test functions, re-reading the neighbours' coefficients
// (cell-centric face loop: no atomics, deterministic).
//
//   OP_DIV  b = -C(q,u)                   (Sec. 4.2, velocity divergence; {{u}} = u^- on walls)
//   OP_CONV y = F^c(v,u), LF flux         (Sec. 4.2, convective term; mirror state on walls)
//   OP_VISC y = -F^nu(vbar,v~;ubar,u~)    (eq. viscous_multiscale, harmweights, minvt)
//   OP_LAP  y = A_L p, SIPG               (eq. ipflux; curved cells only, boxes use laplace_box.cu)
//   OP_MASS y = M(v,u) = (v,u)            (Sec. 4.2 mass term; volume only, enriched DoFs included)
//   OP_DIVDIV y = D(v,u) = (div v, tau_D div u) (eq. div-div; volume only, tau_D per cell in m.tau_d)
//
// Wall-layer cells add the enrichment u~ = psi sum_B N_B u~_B (eq. enrichment) at q_wall
// wall-normal Gauss points, with psi and grad psi read from the wall tables.
//
// Geometry: GEO_BOX cells are axis-aligned boxes (diagonal Jacobian from the row spacing);
// GEO_CURVED cells are isoparametric Q_k images of the reference cube (the periodic-hill setting of
// Sec. 5.2, the mesh "mapped onto the exact ... geometry using the same polynomial ansatz"), with
// J^-1 and det J read per quadrature point from the metric tables.
//
// Every sum-factorisation phase is batched over the velocity components, over both faces normal
// to one direction and over both sides of those faces, so one barrier separates phases that each
// carry enough independent outputs to occupy the CTA (about 35 barriers per cell).
#include <type_traits>

#include "df64.cuh"
#include "metric.cuh"
#include "sumfac.cuh"

namespace dgw {

template <typename T>
__device__ __forceinline__ T cell_h(const MeshView<T> &m, int c, int d) {
  if (d == 0) return m.hx;
  if (d == 2) return m.hz;
  return m.hy[(c / m.nx) % m.ny];
}

template <typename T>
__device__ void load_basis(const Basis<T> *g, Basis<T> *s) {
  const int words = sizeof(Basis<T>) / sizeof(int);
  const int *src = reinterpret_cast<const int *>(g);
  int *dst = reinterpret_cast<int *>(s);
  for (int t = threadIdx.x; t < words; t += blockDim.x) dst[t] = src[t];
}

// One term or the sum of two terms (same output shape) of a 1-D pass.
template <typename T>
struct Pass {
  const T *in;
  const T *M;
  const T *in2;
  const T *M2;
  T *out;
};

// nb independent passes along axis ax over arrays of input dims (s0, s1, s2); desc(b) returns the
// b-th pass. Matrices are stored q x n (points x nodes): forward maps nodes -> points, trans maps
// points -> nodes. acc adds into the output. Ends with a barrier.
template <typename T, typename F>
__device__ void pass_batch(F desc, int nb, int s0, int s1, int s2, int ax, int n, int q, bool trans, bool acc) {
  const int mi = trans ? q : n, mo = trans ? n : q;
  const int o0 = ax == 0 ? mo : s0, o1 = ax == 1 ? mo : s1, o2 = ax == 2 ? mo : s2;
  const int size = o0 * o1 * o2;
  const int stride = ax == 0 ? 1 : (ax == 1 ? s0 : s0 * s1);
  for (int t = threadIdx.x; t < nb * size; t += blockDim.x) {
    const int b = t / size, e = t - b * size;
    const int i0 = e % o0, i1 = (e / o0) % o1, i2 = e / (o0 * o1);
    const int r = ax == 0 ? i0 : (ax == 1 ? i1 : i2);
    const int base = (ax == 0 ? 0 : i0) + s0 * ((ax == 1 ? 0 : i1) + s1 * (ax == 2 ? 0 : i2));
    const Pass<T> d = desc(b);
    T sum = T(0);
    if (!trans) {
      const T *row = d.M + r * n;
      for (int c = 0; c < mi; ++c) sum += row[c] * d.in[base + c * stride];
      if (d.in2) {
        const T *row2 = d.M2 + r * n;
        for (int c = 0; c < mi; ++c) sum += row2[c] * d.in2[base + c * stride];
      }
    } else {
      for (int c = 0; c < mi; ++c) sum += d.M[c * n + r] * d.in[base + c * stride];
      if (d.in2)
        for (int c = 0; c < mi; ++c) sum += d.M2[c * n + r] * d.in2[base + c * stride];
    }
    d.out[e] = acc ? d.out[e] + sum : sum;
  }
  __syncthreads();
}

// Trilinear weight N_v and its reference gradient at a point from the 1-D factors
// f[d][0] = 1 - xi_d, f[d][1] = xi_d.
template <typename T>
__device__ __forceinline__ void q1_vertex(const T f[3][2], int v, T &N, T dN[3]) {
  const int b0 = v & 1, b1 = (v >> 1) & 1, b2 = (v >> 2) & 1;
  const T s0 = b0 ? T(1) : T(-1), s1 = b1 ? T(1) : T(-1), s2 = b2 ? T(1) : T(-1);
  const T f12 = f[1][b1] * f[2][b2];
  N = f[0][b0] * f12;
  dN[0] = s0 * f12;
  dN[1] = s1 * f[0][b0] * f[2][b2];
  dN[2] = s2 * f[0][b0] * f[1][b1];
}

// Adds to out[24] the sum over npts points of 24 per-point contributions (the enriched test
// functions e_a psi N_v, output a * 8 + v). Each thread accumulates its points in registers; a
// butterfly reduce-scatter halves the set a lane holds at each of three steps (27 shuffles per warp
// instead of 24 x 5), and one pass adds the warps' partial sums in a fixed order. part holds
// 24 T per warp. Ends with a barrier.
template <typename T, typename F>
__device__ void reduce24(int npts, F contrib, T *out, T *part) {
  T acc[24];
#pragma unroll
  for (int o = 0; o < 24; ++o) acc[o] = T(0);
  for (int p = threadIdx.x; p < npts; p += blockDim.x) contrib(p, acc);
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  {
    const bool up = lane & 16;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const T send = up ? acc[i] : acc[i + 12], keep = up ? acc[i + 12] : acc[i];
      acc[i] = keep + __shfl_xor_sync(full, send, 16);
    }
  }
  {
    const bool up = lane & 8;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const T send = up ? acc[i] : acc[i + 6], keep = up ? acc[i + 6] : acc[i];
      acc[i] = keep + __shfl_xor_sync(full, send, 8);
    }
  }
  {
    const bool up = lane & 4;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const T send = up ? acc[i] : acc[i + 3], keep = up ? acc[i + 3] : acc[i];
      acc[i] = keep + __shfl_xor_sync(full, send, 4);
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    acc[i] += __shfl_xor_sync(full, acc[i], 2);
    acc[i] += __shfl_xor_sync(full, acc[i], 1);
  }
  if ((lane & 3) == 0) {
    const int base = ((lane & 16) ? 12 : 0) + ((lane & 8) ? 6 : 0) + ((lane & 4) ? 3 : 0);
    for (int i = 0; i < 3; ++i) part[warp * 24 + base + i] = acc[i];
  }
  __syncthreads();
  if (threadIdx.x < 24) {
    T sum = T(0);
    for (int w = 0; w < nw; ++w) sum += part[w * 24 + threadIdx.x];
    out[threadIdx.x] += sum;
  }
  __syncthreads();
}

// The same for the 3 enriched test functions psi e_a of the constant weight (l = 0): plain warp
// sums, then the warps' partial sums in a fixed order. part holds 3 T per warp. Ends with a barrier.
template <typename T, typename F>
__device__ void reduce3(int npts, F contrib, T *out, T *part) {
  T acc[3] = {T(0), T(0), T(0)};
  for (int p = threadIdx.x; p < npts; p += blockDim.x) contrib(p, acc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off);
  if (lane == 0)
    for (int i = 0; i < 3; ++i) part[warp * 3 + i] = acc[i];
  __syncthreads();
  if (threadIdx.x < 3) {
    T sum = T(0);
    for (int w = 0; w < nw; ++w) sum += part[w * 3 + threadIdx.x];
    out[threadIdx.x] += sum;
  }
  __syncthreads();
}

// Enriched test-function integrals over npts points into out: contrib(p, acc, NV) adds the
// contributions of point p for NV weights per component (8: the trilinear weights of l = 1, output
// a * 8 + v; 1: the constant weight of l = 0, output a).
template <typename T, typename F>
__device__ __forceinline__ void reduce_enr(bool l0, int npts, F contrib, T *out, T *part) {
  if (l0) reduce3<T>(npts, [&](int p, T *acc) { contrib(p, acc, std::integral_constant<int, 1>{}); }, out, part);
  else reduce24<T>(npts, [&](int p, T *acc) { contrib(p, acc, std::integral_constant<int, 8>{}); }, out, part);
}


// Value and reference gradient of the enrichment weight v of NV at the point (l = 0: 1 and 0).
template <typename T, int NV>
__device__ __forceinline__ void enr_weight(const T f[3][2], int v, T &Nv, T dN[3]) {
  if (NV == 1) {
    Nv = T(1);
    dN[0] = dN[1] = dN[2] = T(0);
  } else {
    q1_vertex(f, v, Nv, dN);
  }
}

// Shared-memory plan (in T words) for one cell. The volume and face phases share one work
// region; inside the face region the neighbour coefficients share room with the arrays written
// after the layer traces are taken, and the integration arrays with the trace arrays.
struct VecPlan {
  int n, n3, qi, qy, P, FP, pn;   // pn = largest (face points along t1) x n
  int uo, r, eo, re, en, part, work, total;
  int vA, vB, vV, vG, vGt, vol_end;                                               // volume regions
  int fV2, fN2, fA0, fA1, fB0, fTr, fC, fE, fUn, fI0, fI1, fI2, fF2, fG2, face_end;  // face regions
};

__host__ __device__ inline VecPlan vec_plan(int op, bool curved, int n, int qin, int qw) {
  VecPlan p;
  if (op == OP_LAP) qw = qin;   // the Laplacian has no enriched point sets
  const bool grad = op == OP_VISC || op == OP_LAP || op == OP_DIVDIV;
  const int nin = op == OP_LAP ? 1 : 3, nout = (op == OP_DIV || op == OP_LAP) ? 1 : 3;
  const int nca = op == OP_LAP ? 1 : ((op == OP_DIV && !curved) ? 1 : 3);
  const int ns = 4 * nca;
  p.n = n;
  p.n3 = n * n * n;
  p.qi = qin;
  p.qy = qw > qin ? qw : qin;
  p.P = qin * p.qy * qin;
  p.FP = qin * p.qy;
  p.pn = p.qy * n;
  const int nn = n * n;
  const int SX = qin * nn, SZ = qin * p.qy * n;
  const int ka = (grad ? 2 : 1) * nin > 2 * nout ? (grad ? 2 : 1) * nin : 2 * nout;
  const int kb = (grad ? 3 : 1) * nin > 3 * nout ? (grad ? 3 : 1) * nin : 3 * nout;
  int o = 0;
  p.uo = o; o += nin * p.n3;
  p.r = o; o += nout * p.n3;
  p.eo = o; o += 24;
  p.re = o; o += 24;
  p.en = o; o += 48;   // enrichment coefficients of the two neighbours of one direction
  p.part = o; o += 4 * 24;   // per-warp partial sums of the enriched reductions (128 threads)
  p.work = o;
  int v = o;
  // the point values V (written by the last forward pass, read until the enriched reduction) share
  // room with A, which is dead between the second forward pass and the second integration pass
  const bool has_v = op == OP_DIV || op == OP_CONV || op == OP_MASS || op == OP_CFL;
  p.vA = v; v += (has_v && 3 * p.P > ka * SX) ? 3 * p.P : ka * SX;
  p.vV = p.vA;
  p.vB = v; v += kb * SZ;
  p.vG = v; v += (op == OP_CONV || op == OP_VISC || op == OP_DIVDIV ? 9 : 3) * p.P;
  p.vGt = v; v += op == OP_VISC ? 9 * p.P : (op == OP_DIVDIV ? p.P : 0);
  p.vol_end = v;
  int f = o;   // trace slots: 2 faces x 2 sides x nca components
  p.fV2 = f; f += ns * nn;
  p.fN2 = f; f += grad ? ns * nn : 0;
  p.fA0 = f; f += ns * p.pn;
  p.fA1 = f; f += grad ? ns * p.pn : 0;
  p.fB0 = f; f += grad ? ns * p.pn : 0;
  p.fTr = f; f += ns * 4 * p.FP;     // value, d/dxi_d, d/dxi_t1, d/dxi_t2
  p.fC = f; f += 2 * 3 * 4 * p.FP;   // coefficients of the standard test functions (face, component)
  p.fE = f; f += (op == OP_CONV || op == OP_VISC) ? 2 * 3 * 4 * p.FP : 0;   // enriched test functions
  p.face_end = f;
  // both neighbours' coefficients: dead once the layers are taken (only en must survive)
  p.fUn = p.fA0;
  if (p.fUn + 2 * nin * p.n3 > p.face_end) p.face_end = p.fUn + 2 * nin * p.n3;
  // integration arrays: written after the traces are consumed, must not reach the coefficients C
  const int isz = 2 * nout * (3 * p.pn + 2 * nn);
  int g = p.fV2 + isz <= p.fC ? p.fV2 : p.face_end;
  p.fI0 = g; g += 2 * nout * p.pn;
  p.fI1 = g; g += 2 * nout * p.pn;
  p.fI2 = g; g += 2 * nout * p.pn;
  p.fF2 = g; g += 2 * nout * nn;
  p.fG2 = g; g += 2 * nout * nn;
  if (g > p.face_end) p.face_end = g;
  if (op == OP_MASS || op == OP_DIVDIV || op == OP_CFL) p.face_end = p.work;   // no face terms
  p.total = p.vol_end > p.face_end ? p.vol_end : p.face_end;
  return p;
}

// in-plane point count the shared-memory plan must hold: the wall set in wall cells under the q_w^3 rule
template <typename T>
__host__ __device__ inline int plan_qin(const MeshView<T> &m, int qset) {
  return m.full_q && m.q[QSET_WALL] > m.q[qset] ? m.q[QSET_WALL] : m.q[qset];
}

// NC > 0: the node count per direction as a compile-time constant (the curved Laplacian, whose point
// sets are all k+1 Gauss points, is instantiated per degree so the pass index arithmetic folds).
// One CTA per cell of rows [0, rb) and [rt, ny) (rb = rt = ny: every row), x fastest.
template <typename T, int OP, int GEO, int NC = 0>
__global__ void __launch_bounds__(128) vector_op_kernel(MeshView<T> m, const T *__restrict__ u, T *__restrict__ y,
                                                        LapEpi<T> epi, int rb, int rt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Basis<T> &B = *reinterpret_cast<Basis<T> *>(smem_raw);
  T *S0 = reinterpret_cast<T *>(smem_raw + ((sizeof(Basis<T>) + 15) / 16) * 16);
  load_basis(m.basis, &B);
  constexpr bool CURVED = GEO == GEO_CURVED;
  constexpr bool GRAD = OP == OP_VISC || OP == OP_LAP || OP == OP_DIVDIV;
  constexpr int NIN = OP == OP_LAP ? 1 : 3;                             // input components
  constexpr int NOUT = (OP == OP_DIV || OP == OP_LAP) ? 1 : 3;          // output components
  const int n = NC > 0 ? NC : m.n1, nn = n * n;
  const int qset = OP == OP_CONV ? QSET_CONV : QSET_LIN;
  const int opc = OP == OP_CONV ? 1 : 0;   // wall-table class
  const VecPlan L = vec_plan(OP, CURVED, n, NC > 0 ? NC : plan_qin(m, qset), NC > 0 ? NC : m.q[QSET_WALL]);
  const int n3 = L.n3;
  T *uo = S0 + L.uo, *r = S0 + L.r, *eo = S0 + L.eo, *re = S0 + L.re, *un = S0 + L.fUn, *en = S0 + L.en;
  int c;
  {
    const int nr = rb + (m.ny - rt), b = blockIdx.x;
    const int i = b % m.nx, r = (b / m.nx) % nr, kz = b / (m.nx * nr);
    c = i + m.nx * ((r < rb ? r : rt + (r - rb)) + m.ny * kz);
  }
  const int ec = OP == OP_LAP ? -1 : m.enr[c];
  const bool enr_c = ec >= 0;
  const bool l0 = m.nef == 1;   // constant enrichment weight: 3 test functions psi e_a per cell
  const T nu = m.visc;
  const int col = CURVED ? metric_col(m, c) : 0;
  for (int t = threadIdx.x; t < NIN * n3; t += blockDim.x) uo[t] = u[(size_t)c * NIN * n3 + t];
  for (int t = threadIdx.x; t < NOUT * n3; t += blockDim.x) r[t] = T(0);
  // enrichment coefficients as 8 trilinear weights per component; with l = 0 the single coefficient
  // is replicated (sum_B N_B = 1 makes that the same field)
  for (int t = threadIdx.x; t < 24; t += blockDim.x) {
    eo[t] = enr_c ? u[3 * m.np + (size_t)ec * 3 * m.nef + (m.nef == 8 ? t : t >> 3)] : T(0);
    re[t] = T(0);
  }
  __syncthreads();
  T h[3] = {T(1), T(1), T(1)};
  if (!CURVED) { h[0] = m.hx; h[1] = m.hy[(c / m.nx) % m.ny]; h[2] = m.hz; }
  const T hinv[3] = {T(1) / h[0], T(1) / h[1], T(1) / h[2]};
  const bool fq = enr_c && m.full_q;   // the paper's q_w^3 rule in wall cells
  const int sets[3] = {fq ? QSET_WALL : qset, enr_c ? QSET_WALL : qset, fq ? QSET_WALL : qset};
  const int q0 = NC > 0 ? NC : B.q[sets[0]], q1 = NC > 0 ? NC : B.q[sets[1]], q2 = NC > 0 ? NC : B.q[sets[2]];
  const int P = q0 * q1 * q2;
  const T vol = h[0] * h[1] * h[2];
  const T *wtv = enr_c ? m.wt_vol[opc] + (size_t)ec * m.nvol[opc] * WT : nullptr;
  const T *S_[3] = {B.S[sets[0]], B.S[sets[1]], B.S[sets[2]]};
  const T *D_[3] = {B.D[sets[0]], B.D[sets[1]], B.D[sets[2]]};
  // metric at volume point (i0, i1): J^-1 and the volume weight dV
  auto vol_metric = [&](int i0, int i1, int i2, T Ji[3][3], T &dV) {
    const T w3 = B.w[sets[0]][i0] * B.w[sets[1]][i1] * B.w[sets[2]][i2];
    if (CURVED) {
      T det;
      load_rec(vol_rec(m, B, col, sets[0], sets[1], i0, i1), Ji, det);
      dV = fabs(det) * w3;
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Ji[a][b] = a == b ? hinv[a] : T(0);
      dV = vol * w3;
    }
  };

  // ================= volume =================
  {
    T *A = S0 + L.vA, *Bv = S0 + L.vB, *V = S0 + L.vV, *G = S0 + L.vG, *Gt = S0 + L.vGt;
    const int SX = q0 * nn, SZ = q0 * q1 * n;
    // P1: X0_a = S_x u_a (and X1_a = D_x u_a for gradients)
    pass_batch<T>([&](int b) -> Pass<T> {
      const int a = b % NIN, k = b / NIN;
      return {uo + a * n3, k ? D_[0] : S_[0], nullptr, nullptr, A + b * SX};
    }, (GRAD ? 2 : 1) * NIN, n, n, n, 0, n, q0, false, false);
    // P2: Y00_a = S_y X0_a (Y01_a = D_y X0_a, Y10_a = S_y X1_a)
    pass_batch<T>([&](int b) -> Pass<T> {
      const int a = b % NIN, k = b / NIN;   // k: 0 Y00, 1 Y01, 2 Y10
      return {A + (k == 2 ? NIN + a : a) * SX, k == 1 ? D_[1] : S_[1], nullptr, nullptr, Bv + b * SZ};
    }, (GRAD ? 3 : 1) * NIN, q0, n, n, 1, n, q1, false, false);
    // P3: values (DIV, CONV) or reference gradients (VISC, LAP) at the points
    pass_batch<T>([&](int b) -> Pass<T> {
      const int a = b % NIN, k = b / NIN;
      if (!GRAD) return {Bv + a * SZ, S_[2], nullptr, nullptr, V + a * P};
      // k = 0: d/dz from Y00; 1: d/dy from Y01; 2: d/dx from Y10
      return {Bv + b * SZ, k == 0 ? D_[2] : S_[2], nullptr, nullptr, G + (a * 3 + 2 - k) * P};
    }, (GRAD ? 3 : 1) * NIN, q0, q1, n, 2, n, q2, false, false);
    T cfl_max = T(0);   // OP_CFL: this thread's largest rate
    // P4: pointwise test-function coefficients (H_{a,d} multiplies d phi / d xi_d)
    const T *nutv = (OP == OP_VISC && enr_c) ? m.nut_vol + (size_t)ec * m.nvol[0] : nullptr;
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
      const int i0 = t % q0, i1 = (t / q0) % q1, i2 = t / (q0 * q1);
      T dV, Ji[3][3];
      if (CURVED) {
        vol_metric(i0, i1, i2, Ji, dV);
      } else {
        dV = vol * B.w[sets[0]][i0] * B.w[sets[1]][i1] * B.w[sets[2]][i2];
      }
      // enrichment at the point: sN_a = sum_v N_v e_av, sD_ad = sum_v dN_v/dxi_d e_av
      T sN[3] = {0, 0, 0}, sD[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      const T *w = nullptr;
      if (enr_c) {
        const T xi[3] = {B.x[sets[0]][i0], B.x[sets[1]][i1], B.x[sets[2]][i2]};
        const T f[3][2] = {{T(1) - xi[0], xi[0]}, {T(1) - xi[1], xi[1]}, {T(1) - xi[2], xi[2]}};
#pragma unroll
        for (int a = 0; a < 3; ++a) enr_trial<T, GRAD>(f, eo + a * 8, l0, sN[a], sD[a]);
        w = wtv + t * WT;
      }
      if (OP == OP_DIV || OP == OP_CONV || OP == OP_MASS || OP == OP_CFL) {
        T uu[3] = {V[t], V[P + t], V[2 * P + t]};
        if (enr_c)
          for (int a = 0; a < 3; ++a) {
            uu[a] += w[0] * sN[a];
            V[a * P + t] = uu[a];
          }
        if (OP == OP_CFL) {   // |J^-1 u|_2: the velocity in reference-cell lengths per unit time
          T cf[3];
          if (CURVED) phys_to_ref(Ji, uu, cf);
          else for (int d = 0; d < 3; ++d) cf[d] = uu[d] * hinv[d];
          cfl_max = max(cfl_max, sqrt(cf[0] * cf[0] + cf[1] * cf[1] + cf[2] * cf[2]));
          continue;
        }
        if (OP == OP_MASS) {   // value coefficients of the test functions
          for (int a = 0; a < 3; ++a) G[a * P + t] = dV * uu[a];
        } else if (CURVED) {
          T cf[3];
          if (OP == OP_DIV) {
            phys_to_ref(Ji, uu, cf);
            for (int d = 0; d < 3; ++d) G[d * P + t] = dV * cf[d];
          } else {
            phys_to_ref(Ji, uu, cf);   // J^-1 u: the convective coefficient is -dV u_a (J^-1 u)_d
            for (int a = 0; a < 3; ++a)
              for (int d = 0; d < 3; ++d) G[(a * 3 + d) * P + t] = -dV * uu[a] * cf[d];
          }
        } else if (OP == OP_DIV) {
          for (int d = 0; d < 3; ++d) G[d * P + t] = dV * uu[d] * hinv[d];
        } else {
          T sd[3];   // -dV u_d / h_d, shared by the three outputs
          for (int d = 0; d < 3; ++d) sd[d] = -dV * uu[d] * hinv[d];
          for (int a = 0; a < 3; ++a)
            for (int d = 0; d < 3; ++d) G[(a * 3 + d) * P + t] = uu[a] * sd[d];
        }
      } else if (OP == OP_LAP) {
        const T gr[3] = {G[t], G[P + t], G[2 * P + t]};
        T g[3], cf[3];
        ref_to_phys(Ji, gr, g);
        phys_to_ref(Ji, g, cf);
        for (int d = 0; d < 3; ++d) G[d * P + t] = dV * cf[d];
      } else {
        T gb[3][3], tb[3][3];
        for (int a = 0; a < 3; ++a) {
          if (CURVED) {
            const T gr[3] = {G[(a * 3) * P + t], G[(a * 3 + 1) * P + t], G[(a * 3 + 2) * P + t]};
            ref_to_phys(Ji, gr, gb[a]);
          } else {
            for (int d = 0; d < 3; ++d) gb[a][d] = G[(a * 3 + d) * P + t] * hinv[d];
          }
        }
        if (OP == OP_DIVDIV) {
          // tau_D div u, with the enrichment's divergence sum_a d(psi sum_v N_v e_av)/dx_a
          T dv = gb[0][0] + gb[1][1] + gb[2][2];
          if (enr_c)
            for (int a = 0; a < 3; ++a) {
              T g[3];
              if (CURVED) ref_to_phys(Ji, sD[a], g);
              dv += w[0] * (CURVED ? g[a] : sD[a][a] * hinv[a]) + sN[a] * w[1 + a];
            }
          const T fd = m.tau_d[c] * dv;
          for (int a = 0; a < 3; ++a)
            for (int d = 0; d < 3; ++d) tb[a][d] = a == d ? fd : T(0);
          Gt[t] = dV * fd;
        } else {
        for (int a = 0; a < 3; ++a)
          for (int d = 0; d < 3; ++d) tb[a][d] = nu * (gb[a][d] + gb[d][a]);
        if (enr_c) {
          T gt[3][3];
          for (int a = 0; a < 3; ++a) {
            if (CURVED) ref_to_phys(Ji, sD[a], gt[a]);
            for (int d = 0; d < 3; ++d) {
              gt[a][d] = w[0] * (CURVED ? gt[a][d] : sD[a][d] * hinv[d]) + sN[a] * w[1 + d];
              Gt[(a * 3 + d) * P + t] = gt[a][d];
            }
          }
          const T nut = nutv[t];
          const T nuh = min(nu + nut, T(2) * sqrt(nu * (nu + nut)));   // eq. (minvt)
          for (int a = 0; a < 3; ++a)
            for (int d = 0; d < 3; ++d) tb[a][d] += nuh * (gt[a][d] + gt[d][a]);
        }
        }
        for (int a = 0; a < 3; ++a) {
          if (CURVED) {
            T cf[3];
            phys_to_ref(Ji, tb[a], cf);
            for (int d = 0; d < 3; ++d) G[(a * 3 + d) * P + t] = dV * cf[d];
          } else {
            for (int d = 0; d < 3; ++d) G[(a * 3 + d) * P + t] = dV * tb[a][d] * hinv[d];
          }
        }
      }
    }
    __syncthreads();
    if constexpr (OP == OP_CFL) {
      // the block's largest rate, then one atomic maximum on the bit pattern (non-negative doubles
      // order like their bits)
      __shared__ T wmax[4];
      for (int off = 16; off > 0; off >>= 1) cfl_max = max(cfl_max, __shfl_xor_sync(0xffffffffu, cfl_max, off));
      if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = cfl_max;
      __syncthreads();
      if (threadIdx.x == 0) {
        T b = wmax[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = max(b, wmax[w]);
        atomicMax(reinterpret_cast<unsigned long long *>(y), (unsigned long long)__double_as_longlong((double)b));
      }
      return;
    }
    // enriched test functions: -(grad(psi N_v) e_a, u x u), (eps(psi N_v e_a), 2(nu+nu_t) eps(u~)) or
    // (div(psi N_v e_a), tau_D div u)
    if (enr_c && (OP == OP_CONV || OP == OP_VISC || OP == OP_DIVDIV)) {
      auto contrib = [&](int t, T *acc, auto nvc) {
        constexpr int NV = decltype(nvc)::value;
        const int i0 = t % q0, i1 = (t / q0) % q1, i2 = t / (q0 * q1);
        const T xi[3] = {B.x[sets[0]][i0], B.x[sets[1]][i1], B.x[sets[2]][i2]};
        const T f[3][2] = {{T(1) - xi[0], xi[0]}, {T(1) - xi[1], xi[1]}, {T(1) - xi[2], xi[2]}};
        const T *w = wtv + t * WT;
        T dV, Ji[3][3];
        if (CURVED) vol_metric(i0, i1, i2, Ji, dV);
        else dV = vol * B.w[sets[0]][i0] * B.w[sets[1]][i1] * B.w[sets[2]][i2];
        T cf[3][3];   // coefficient of d(psi N_v)/dx_d in output (a, v)
        T beta[3], alpha[3][3];
        if (OP == OP_CONV) {
          // cf_ad = -dV u_a u_d has rank one: beta_a = u_a (-dV u . grad psi), alpha_a = u_a (-dV psi J^-1 u)
          const T uu[3] = {V[t], V[P + t], V[2 * P + t]};
          const T bs = -dV * (uu[0] * w[1] + uu[1] * w[2] + uu[2] * w[3]);
          T av[3] = {T(0), T(0), T(0)};
          if (NV == 8) {
            const T pw = -dV * w[0];
            if (CURVED) {
              phys_to_ref(Ji, uu, av);
#pragma unroll
              for (int e = 0; e < 3; ++e) av[e] *= pw;
            } else {
#pragma unroll
              for (int e = 0; e < 3; ++e) av[e] = pw * uu[e] * hinv[e];
            }
          }
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            beta[a] = uu[a] * bs;
#pragma unroll
            for (int e = 0; e < 3; ++e) alpha[a][e] = uu[a] * av[e];
          }
        } else if (OP == OP_DIVDIV) {
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int d = 0; d < 3; ++d) cf[a][d] = a == d ? Gt[t] : T(0);
        } else {
          const T nd = dV * (nu + nutv[t]);
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int d = 0; d < 3; ++d) cf[a][d] = nd * (Gt[(a * 3 + d) * P + t] + Gt[(d * 3 + a) * P + t]);
        }
        // grad(psi N_v) = psi grad N_v + N_v grad psi: the coefficient of N_v is beta_a = cf_a . grad psi,
        // that of dN_v/dxi_e is alpha_a[e] = psi (J^-1 cf_a)_e
#pragma unroll
        for (int a = 0; a < 3 && OP != OP_CONV; ++a) {
          beta[a] = cf[a][0] * w[1] + cf[a][1] * w[2] + cf[a][2] * w[3];
          if (NV == 8) {
            if (CURVED) {
              phys_to_ref(Ji, cf[a], alpha[a]);
#pragma unroll
              for (int e = 0; e < 3; ++e) alpha[a][e] *= w[0];
            } else {
#pragma unroll
              for (int e = 0; e < 3; ++e) alpha[a][e] = w[0] * cf[a][e] * hinv[e];
            }
          }
        }
        if (NV == 1) {
#pragma unroll
          for (int a = 0; a < 3; ++a) acc[a] += beta[a];
        } else {
          acc_trilinear<T>(f, beta, alpha, acc);
        }
      };
      reduce_enr<T>(l0, P, contrib, re, S0 + L.part);
    }
    if (OP == OP_MASS) {
      // enriched test functions: (psi N_v e_a, u)
      if (enr_c) {
        auto contrib = [&](int t, T *acc, auto nvc) {
          constexpr int NV = decltype(nvc)::value;
          const int i0 = t % q0, i1 = (t / q0) % q1, i2 = t / (q0 * q1);
          const T xi[3] = {B.x[sets[0]][i0], B.x[sets[1]][i1], B.x[sets[2]][i2]};
          const T f[3][2] = {{T(1) - xi[0], xi[0]}, {T(1) - xi[1], xi[1]}, {T(1) - xi[2], xi[2]}};
          const T psi = wtv[t * WT];
          const T pv[3] = {psi * G[t], psi * G[P + t], psi * G[2 * P + t]};   // dV psi u_a
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            T Nv, dN[3];
            enr_weight<T, NV>(f, v, Nv, dN);
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[a * NV + v] += Nv * pv[a];
          }
        };
        reduce_enr<T>(l0, P, contrib, re, S0 + L.part);
      }
      // integrate the value coefficients back to the nodes: S_z^T, S_y^T, S_x^T
      pass_batch<T>([&](int a) -> Pass<T> {
        return {G + a * P, S_[2], nullptr, nullptr, Bv + a * SZ};
      }, 3, q0, q1, q2, 2, n, q2, true, false);
      pass_batch<T>([&](int a) -> Pass<T> {
        return {Bv + a * SZ, S_[1], nullptr, nullptr, A + a * SX};
      }, 3, q0, q1, n, 1, n, q1, true, false);
      pass_batch<T>([&](int a) -> Pass<T> {
        return {A + a * SX, S_[0], nullptr, nullptr, r + a * n3};
      }, 3, q0, n, n, 0, n, q0, true, true);
    } else {
    // P5-P7: integrate the gradient coefficients back to the nodes (z, y, x)
    pass_batch<T>([&](int b) -> Pass<T> {
      const int a = b % NOUT, k = b / NOUT;   // k: 0 Z0 = D_z^T H_z, 1 Z1 = S_z^T H_y, 2 Z2 = S_z^T H_x
      return {G + (a * 3 + 2 - k) * P, k == 0 ? D_[2] : S_[2], nullptr, nullptr, Bv + b * SZ};
    }, 3 * NOUT, q0, q1, q2, 2, n, q2, true, false);
    pass_batch<T>([&](int b) -> Pass<T> {
      const int a = b % NOUT, k = b / NOUT;   // k: 0 Y0 = S_y^T Z0 + D_y^T Z1, 1 Y1 = S_y^T Z2
      if (k == 0) return {Bv + a * SZ, S_[1], Bv + (NOUT + a) * SZ, D_[1], A + b * SX};
      return {Bv + (2 * NOUT + a) * SZ, S_[1], nullptr, nullptr, A + b * SX};
    }, 2 * NOUT, q0, q1, n, 1, n, q1, true, false);
    pass_batch<T>([&](int a) -> Pass<T> {
      return {A + a * SX, S_[0], A + (NOUT + a) * SX, D_[0], r + a * n3};
    }, NOUT, q0, n, n, 0, n, q0, true, true);
    }
  }

  if constexpr (OP != OP_MASS && OP != OP_DIVDIV && OP != OP_CFL) {
  // ================= faces, one direction (two faces) at a time =================
  // trace slots per direction: (face s, side, component); on boxes the divergence needs the normal
  // component only
  constexpr int NCA = OP == OP_LAP ? 1 : ((OP == OP_DIV && !CURVED) ? 1 : 3);
  constexpr int NS = 4 * NCA;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int t1, t2;
    face_axes(d, t1, t2);
    int nbr[2], enb[2];
    bool enr_o[2];
    for (int s = 0; s < 2; ++s) {
      nbr[s] = neighbour(m, c, 2 * d + s);
      enb[s] = (OP != OP_LAP && nbr[s] >= 0) ? m.enr[nbr[s]] : -1;
      enr_o[s] = nbr[s] >= 0 ? enb[s] >= 0 : enr_c;   // the mirror side carries c's class
    }
    // point sets of the faces normal to d: each face takes q_w along its tangential axis y (every
    // tangential axis under the q_w^3 rule) if it touches an enriched cell. When that rule differs
    // between the two faces (the q_w^3 rule above the enriched layer, switched-off columns), the
    // faces are done in two passes, each zeroing the other face's coefficients.
    const bool ef0 = enr_c || enr_o[0], ef1 = enr_c || enr_o[1];
    const int ngrp = ((t1 == 1 || t2 == 1 || m.full_q) && ef0 != ef1) ? 2 : 1;
    for (int grp = 0; grp < ngrp; ++grp) {
    const bool enr_any = ngrp == 2 ? (grp ? ef1 : ef0) : (ef0 || ef1);
    const int s1 = ((t1 == 1 || m.full_q) && enr_any) ? QSET_WALL : qset;
    const int s2 = ((t2 == 1 || m.full_q) && enr_any) ? QSET_WALL : qset;
    const int p1 = NC > 0 ? NC : B.q[s1], p2 = NC > 0 ? NC : B.q[s2], FP = p1 * p2;
    for (int t = threadIdx.x; t < 2 * NIN * n3; t += blockDim.x) {
      const int s = t / (NIN * n3), e = t - s * NIN * n3;
      un[t] = nbr[s] >= 0 ? u[(size_t)nbr[s] * NIN * n3 + e] : T(0);
    }
    for (int t = threadIdx.x; t < 48; t += blockDim.x) {
      const int s = t / 24;
      const int o = t - 24 * s;
      en[t] = enb[s] >= 0 ? u[3 * m.np + (size_t)enb[s] * 3 * m.nef + (m.nef == 8 ? o : o >> 3)] : T(0);
    }
    __syncthreads();
    T *V2 = S0 + L.fV2, *N2 = S0 + L.fN2, *A0 = S0 + L.fA0, *A1 = S0 + L.fA1, *B0 = S0 + L.fB0, *Tr = S0 + L.fTr;
    // slot k = (s * 2 + side) * NCA + a; side 0 = own cell at xi_d = s, side 1 = neighbour at xi_d = 1 - s
    // T1: face-layer values and reference normal derivatives
    for (int t = threadIdx.x; t < NS * nn; t += blockDim.x) {
      const int k = t / nn, node = t - k * nn;
      const int a = NCA == 1 ? (OP == OP_DIV ? d : 0) : k % NCA, side = (k / NCA) % 2, s = k / (2 * NCA);
      const T *src = side ? un + (s * NIN + a) * n3 : uo + a * n3;
      const int ep = side ? 1 - s : s;
      const int i1 = node % n, i2 = node / n;
      V2[t] = src[node_index(d, t1, t2, ep ? n - 1 : 0, i1, i2, n)];
      if (GRAD) {
        T sum = T(0);
        for (int j = 0; j < n; ++j) sum += B.dend[ep][j] * src[node_index(d, t1, t2, j, i1, i2, n)];
        N2[t] = sum;
      }
    }
    __syncthreads();
    // T2: along t1 (n -> p1)
    pass_batch<T>([&](int b) -> Pass<T> {
      const int k = b % NS, j = b / NS;   // j: 0 A0 = S1 V2, 1 A1 = D1 V2, 2 B0 = S1 N2
      const T *in = (j == 2 ? N2 : V2) + k * nn;
      T *out = (j == 0 ? A0 : (j == 1 ? A1 : B0)) + k * L.pn;
      return {in, j == 1 ? B.D[s1] : B.S[s1], nullptr, nullptr, out};
    }, GRAD ? 3 * NS : NS, n, n, 1, 0, n, p1, false, false);
    // T3: along t2 (n -> p2): value, d/dxi_d, d/dxi_t1, d/dxi_t2 at the face points
    pass_batch<T>([&](int b) -> Pass<T> {
      const int k = b % NS, j = b / NS;   // j: 0 val = S2 A0, 1 gd = S2 B0, 2 gt1 = S2 A1, 3 gt2 = D2 A0
      const T *in = (j == 1 ? B0 : (j == 2 ? A1 : A0)) + k * L.pn;
      return {in, j == 3 ? B.D[s2] : B.S[s2], nullptr, nullptr, Tr + (k * 4 + j) * L.FP};
    }, GRAD ? 4 * NS : NS, p1, n, 1, 1, n, p2, false, false);
    // pointwise fluxes -> coefficients of the own test functions
    T *C = S0 + L.fC, *E = S0 + L.fE;
    T hinv_nb1[2];   // the y-spacing of each neighbour, inverted once (walls: the own)
#pragma unroll
    for (int s = 0; s < 2; ++s) hinv_nb1[s] = (!CURVED && nbr[s] >= 0) ? T(1) / cell_h(m, nbr[s], 1) : hinv[1];
    for (int t = threadIdx.x; t < 2 * FP; t += blockDim.x) {
      const int s = t / FP, pt = t - s * FP;
      if (ngrp == 2 && s != grp) {   // the other face is done in its own pass
        T *Cz = C + s * 3 * 4 * L.FP;
        for (int j = 0; j < 12; ++j) Cz[j * L.FP + pt] = T(0);
        if (OP == OP_CONV || OP == OP_VISC) {
          T *Ez = E + s * 3 * 4 * L.FP;
          for (int j = 0; j < 12; ++j) Ez[j * L.FP + pt] = T(0);
        }
        continue;
      }
      const int f = 2 * d + s, side = s;
      const int nb = nbr[s], eb = enb[s];
      const int a1 = pt % p1, a2 = pt / p1;
      const T sgn = side ? T(1) : T(-1);
      const bool both = enr_c && enr_o[s], iface = enr_c != enr_o[s];
      const T tau = nb >= 0 ? max(m.tau[c], m.tau[nb]) : T(10) * m.tau[c];
      const T *wts = enr_c ? m.wt_face[opc] + (((size_t)ec * 6 + f) * m.fpmax[opc]) * WT : nullptr;
      const T *wto = (nb >= 0 && eb >= 0) ? m.wt_face[opc] + (((size_t)eb * 6 + (f ^ 1)) * m.fpmax[opc]) * WT : nullptr;
      T fs[3][2], fo[3][2];   // 1-D factors of the trilinear weights on both sides
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const T xe = e == d ? T(side) : (e == t1 ? B.x[s1][a1] : B.x[s2][a2]);
        const T xoe = e == d ? T(1 - side) : xe;
        fs[e][0] = T(1) - xe; fs[e][1] = xe;
        fo[e][0] = T(1) - xoe; fo[e][1] = xoe;
      }
      T *Cs = C + s * 3 * 4 * L.FP, *Es = E + s * 3 * 4 * L.FP;
      if constexpr (!CURVED) {
        const T dA = h[t1] * h[t2] * B.w[s1][a1] * B.w[s2][a2];
        T ub_s[3] = {0, 0, 0}, ub_o[3] = {0, 0, 0}, ut_s[3] = {0, 0, 0}, ut_o[3] = {0, 0, 0};
        T gbs[3][3], gbo[3][3], gts[3][3], gto[3][3];
        // the neighbour's inverse spacings (x and z spacings are uniform)
        const T hio[3] = {hinv[0], hinv_nb1[s], hinv[2]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (OP == OP_DIV && a != d) continue;   // the divergence needs the normal component only
          const int ka = NCA == 1 ? 0 : a;
          const T *tr_s = Tr + (((s * 2 + 0) * NCA + ka) * 4) * L.FP;
          const T *tr_o = Tr + (((s * 2 + 1) * NCA + ka) * 4) * L.FP;
          ub_s[a] = tr_s[pt];
          if (GRAD) {
            gbs[a][d] = tr_s[L.FP + pt] * hinv[d];
            gbs[a][t1] = tr_s[2 * L.FP + pt] * hinv[t1];
            gbs[a][t2] = tr_s[3 * L.FP + pt] * hinv[t2];
          }
          // enrichment u~_a = psi sum_v N_v e_av and its physical gradient
          if (enr_c) {
            const T *w = wts + pt * WT;
            T sN, sD[3];
            enr_trial<T, GRAD>(fs, eo + a * 8, l0, sN, sD);
            ut_s[a] = w[0] * sN;
            if (GRAD)
#pragma unroll
              for (int e = 0; e < 3; ++e) gts[a][e] = w[0] * sD[e] * hinv[e] + sN * w[1 + e];
          } else if (GRAD) {
            gts[a][0] = gts[a][1] = gts[a][2] = T(0);
          }
          if (nb >= 0) {
            ub_o[a] = tr_o[pt];
            if (GRAD) {
              gbo[a][d] = tr_o[L.FP + pt] * hio[d];
              gbo[a][t1] = tr_o[2 * L.FP + pt] * hio[t1];
              gbo[a][t2] = tr_o[3 * L.FP + pt] * hio[t2];
            }
            if (wto) {
              const T *w = wto + pt * WT;
              T sN, sD[3];
              enr_trial<T, GRAD>(fo, en + s * 24 + a * 8, l0, sN, sD);
              ut_o[a] = w[0] * sN;
              if (GRAD)
#pragma unroll
                for (int e = 0; e < 3; ++e) gto[a][e] = w[0] * sD[e] * hio[e] + sN * w[1 + e];
            } else if (GRAD) {
              gto[a][0] = gto[a][1] = gto[a][2] = T(0);
            }
          } else {
            // mirror principle on no-slip walls: u+ = -u-, grad u+ = grad u-
            ub_o[a] = -ub_s[a];
            ut_o[a] = -ut_s[a];
            if (GRAD)
#pragma unroll
              for (int e = 0; e < 3; ++e) { gbo[a][e] = gbs[a][e]; gto[a][e] = gts[a][e]; }
          }
        }
        if (OP == OP_DIV) {
          const T us = ub_s[d] + ut_s[d], uo_ = ub_o[d] + ut_o[d];
          const T avg = nb >= 0 ? T(0.5) * (us + uo_) : us;
          Cs[pt] = -dA * sgn * avg;
        } else if (OP == OP_CONV) {
          T um[3], up[3];
          for (int a = 0; a < 3; ++a) { um[a] = ub_s[a] + ut_s[a]; up[a] = ub_o[a] + ut_o[a]; }
          const T unm = sgn * um[d], unp = sgn * up[d];
          const T lam = max(T(2) * fabs(unm), T(2) * fabs(unp));
          for (int a = 0; a < 3; ++a) {
            const T Fa = T(0.5) * (um[a] * unm + up[a] * unp) + T(0.5) * lam * (um[a] - up[a]);
            Cs[(a * 4) * L.FP + pt] = dA * Fa;
            Es[(a * 4) * L.FP + pt] = dA * Fa;
          }
        } else if (OP == OP_VISC) {
          const T *nuts = enr_c ? m.nut_face + ((size_t)ec * 6 + f) * m.fpmax[0] : nullptr;
          const T *nuto = (nb >= 0 && eb >= 0) ? m.nut_face + ((size_t)eb * 6 + (f ^ 1)) * m.fpmax[0] : nullptr;
          const T nut_s = nuts ? nuts[pt] : T(0);
          const T nut_o = nb >= 0 ? (nuto ? nuto[pt] : T(0)) : nut_s;
          T jb[3], jt[3], jtot[3], avgb_n[3], avgt_n[3] = {0, 0, 0};
          for (int a = 0; a < 3; ++a) {
            jb[a] = ub_s[a] - ub_o[a];
            jt[a] = ut_s[a] - ut_o[a];
            jtot[a] = jb[a] + jt[a];
            avgb_n[a] = T(0.5) * nu * sgn * ((gbs[a][d] + gbs[d][a]) + (gbo[a][d] + gbo[d][a]));
          }
          T wt_s = T(0.5);
          if (both) {
            const T den = T(2) * nu + nut_s + nut_o;
            const T iden = T(1) / den;
            wt_s = (nu + nut_o) * iden;
            const T wt_o = (nu + nut_s) * iden;
            for (int a = 0; a < 3; ++a)
              avgt_n[a] = sgn * (wt_s * (nu + nut_s) * (gts[a][d] + gts[d][a]) + wt_o * (nu + nut_o) * (gto[a][d] + gto[d][a]));
          }
          T jadj[3];
          for (int a = 0; a < 3; ++a) jadj[a] = jb[a] + (iface ? jt[a] : T(0));
          for (int a = 0; a < 3; ++a) {
            T cv = -avgb_n[a] + tau * nu * jtot[a];
            if (both) cv -= avgt_n[a];
            // coefficient of phi: dA cv; of dphi/dxi_b: dA nu/2 sgn (jadj_a delta_bd + delta_ad jadj_b) / h_b
            Cs[(a * 4 + 0) * L.FP + pt] = dA * cv;
            Cs[(a * 4 + 1) * L.FP + pt] = dA * T(0.5) * nu * sgn * (jadj[a] + (a == d ? jadj[d] : T(0))) * hinv[d];
            Cs[(a * 4 + 2) * L.FP + pt] = dA * T(0.5) * nu * sgn * (a == d ? jadj[t1] : T(0)) * hinv[t1];
            Cs[(a * 4 + 3) * L.FP + pt] = dA * T(0.5) * nu * sgn * (a == d ? jadj[t2] : T(0)) * hinv[t2];
            if (enr_c) {
              T cve = tau * nu * jtot[a];
              if (both) cve -= avgt_n[a];
              if (iface) cve -= avgb_n[a];
              Es[(a * 4 + 0) * L.FP + pt] = dA * cve;
              for (int b = 0; b < 3; ++b) {
                // (w F^{nu+nut}(v~), [[u~]] + [[ubar]]) on d Omega~_e: physical-gradient coefficient
                const T coef = both ? wt_s * (nu + nut_s) * sgn * ((b == d ? jtot[a] : T(0)) + (a == d ? jtot[b] : T(0))) : T(0);
                Es[(a * 4 + 1 + b) * L.FP + pt] = dA * coef;
              }
            }
          }
        }
      } else {
        // ---- curved cells: metric of both sides at the shared point, outward normal, area weight
        T Js[3][3], Jo[3][3], dets, deto;
        load_rec(face_rec(m, B, col, d, s, s1, s2, a1, a2), Js, dets);
        if (nb >= 0) load_rec(face_rec(m, B, metric_col(m, nb), d, 1 - s, s1, s2, a1, a2), Jo, deto);
        const T nrm = sqrt(Js[d][0] * Js[d][0] + Js[d][1] * Js[d][1] + Js[d][2] * Js[d][2]);
        const T snrm = sgn / nrm;
        const T nv[3] = {snrm * Js[d][0], snrm * Js[d][1], snrm * Js[d][2]};
        const T dA = fabs(dets) * nrm * B.w[s1][a1] * B.w[s2][a2];
        T vJ[3];   // J^-1 n: the normal derivative is grad_xi . (J^-1 n)
        phys_to_ref(Js, nv, vJ);
        T ub_s[3] = {0, 0, 0}, ub_o[3] = {0, 0, 0}, ut_s[3] = {0, 0, 0}, ut_o[3] = {0, 0, 0};
        T gbs[3][3], gbo[3][3], gts[3][3], gto[3][3];
#pragma unroll
        for (int a = 0; a < NIN; ++a) {
          const int ka = NCA == 1 ? 0 : a;
          const T *tr_s = Tr + (((s * 2 + 0) * NCA + ka) * 4) * L.FP;
          const T *tr_o = Tr + (((s * 2 + 1) * NCA + ka) * 4) * L.FP;
          ub_s[a] = tr_s[pt];
          if (GRAD) {
            T gr[3];
            gr[d] = tr_s[L.FP + pt]; gr[t1] = tr_s[2 * L.FP + pt]; gr[t2] = tr_s[3 * L.FP + pt];
            ref_to_phys(Js, gr, gbs[a]);
          }
          if (OP != OP_LAP && enr_c) {
            const T *w = wts + pt * WT;
            T sN, sD[3];
            enr_trial<T, GRAD>(fs, eo + a * 8, l0, sN, sD);
            ut_s[a] = w[0] * sN;
            if (GRAD) {
              T gp[3];
              ref_to_phys(Js, sD, gp);
#pragma unroll
              for (int e = 0; e < 3; ++e) gts[a][e] = w[0] * gp[e] + sN * w[1 + e];
            }
          } else if (GRAD) {
            gts[a][0] = gts[a][1] = gts[a][2] = T(0);
          }
          if (nb >= 0) {
            ub_o[a] = tr_o[pt];
            if (GRAD) {
              T gr[3];
              gr[d] = tr_o[L.FP + pt]; gr[t1] = tr_o[2 * L.FP + pt]; gr[t2] = tr_o[3 * L.FP + pt];
              ref_to_phys(Jo, gr, gbo[a]);
            }
            if (OP != OP_LAP && wto) {
              const T *w = wto + pt * WT;
              T sN, sD[3];
              enr_trial<T, GRAD>(fo, en + s * 24 + a * 8, l0, sN, sD);
              ut_o[a] = w[0] * sN;
              if (GRAD) {
                T gp[3];
                ref_to_phys(Jo, sD, gp);
#pragma unroll
                for (int e = 0; e < 3; ++e) gto[a][e] = w[0] * gp[e] + sN * w[1 + e];
              }
            } else if (GRAD) {
              gto[a][0] = gto[a][1] = gto[a][2] = T(0);
            }
          } else {
            // mirror principle on no-slip walls: u+ = -u-, grad u+ = grad u-
            ub_o[a] = -ub_s[a];
            ut_o[a] = -ut_s[a];
            if (GRAD)
#pragma unroll
              for (int e = 0; e < 3; ++e) { gbo[a][e] = gbs[a][e]; gto[a][e] = gts[a][e]; }
          }
        }
        const int ax[3] = {d, t1, t2};   // reference axis of trace slots 1..3
        if (OP == OP_LAP) {
          // SIPG (eq. ipflux); homogeneous Neumann walls carry no face terms
          T c0 = T(0), cj = T(0);
          if (nb >= 0) {
            const T gn = (gbs[0][0] + gbo[0][0]) * nv[0] + (gbs[0][1] + gbo[0][1]) * nv[1] + (gbs[0][2] + gbo[0][2]) * nv[2];
            const T jump = ub_s[0] - ub_o[0];
            c0 = dA * (T(-0.5) * gn + tau * jump);
            cj = dA * T(-0.5) * jump;
          }
          Cs[pt] = c0;
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) Cs[(1 + jj) * L.FP + pt] = cj * vJ[ax[jj]];
        } else if (OP == OP_DIV) {
          T us = T(0), uo_ = T(0);
#pragma unroll
          for (int e = 0; e < 3; ++e) { us += (ub_s[e] + ut_s[e]) * nv[e]; uo_ += (ub_o[e] + ut_o[e]) * nv[e]; }
          const T avg = nb >= 0 ? T(0.5) * (us + uo_) : us;
          Cs[pt] = -dA * avg;
        } else if (OP == OP_CONV) {
          T um[3], up[3];
          for (int a = 0; a < 3; ++a) { um[a] = ub_s[a] + ut_s[a]; up[a] = ub_o[a] + ut_o[a]; }
          const T unm = um[0] * nv[0] + um[1] * nv[1] + um[2] * nv[2];
          const T unp = up[0] * nv[0] + up[1] * nv[1] + up[2] * nv[2];
          const T lam = max(T(2) * fabs(unm), T(2) * fabs(unp));
          for (int a = 0; a < 3; ++a) {
            const T Fa = T(0.5) * (um[a] * unm + up[a] * unp) + T(0.5) * lam * (um[a] - up[a]);
            Cs[(a * 4) * L.FP + pt] = dA * Fa;
            Es[(a * 4) * L.FP + pt] = dA * Fa;
          }
        } else {  // VISC
          const T *nuts = enr_c ? m.nut_face + ((size_t)ec * 6 + f) * m.fpmax[0] : nullptr;
          const T *nuto = (nb >= 0 && eb >= 0) ? m.nut_face + ((size_t)eb * 6 + (f ^ 1)) * m.fpmax[0] : nullptr;
          const T nut_s = nuts ? nuts[pt] : T(0);
          const T nut_o = nb >= 0 ? (nuto ? nuto[pt] : T(0)) : nut_s;
          T jb[3], jt[3], jtot[3], avgb_n[3], avgt_n[3] = {0, 0, 0};
          for (int a = 0; a < 3; ++a) {
            jb[a] = ub_s[a] - ub_o[a];
            jt[a] = ut_s[a] - ut_o[a];
            jtot[a] = jb[a] + jt[a];
            T sn = T(0);
            for (int e = 0; e < 3; ++e) sn += ((gbs[a][e] + gbs[e][a]) + (gbo[a][e] + gbo[e][a])) * nv[e];
            avgb_n[a] = T(0.5) * nu * sn;
          }
          T wt_s = T(0.5);
          if (both) {
            const T den = T(2) * nu + nut_s + nut_o;
            const T iden = T(1) / den;
            wt_s = (nu + nut_o) * iden;
            const T wt_o = (nu + nut_s) * iden;
            for (int a = 0; a < 3; ++a) {
              T sn = T(0);
              for (int e = 0; e < 3; ++e)
                sn += (wt_s * (nu + nut_s) * (gts[a][e] + gts[e][a]) + wt_o * (nu + nut_o) * (gto[a][e] + gto[e][a])) * nv[e];
              avgt_n[a] = sn;
            }
          }
          T jadj[3];
          for (int a = 0; a < 3; ++a) jadj[a] = jb[a] + (iface ? jt[a] : T(0));
          for (int a = 0; a < 3; ++a) {
            T cv = -avgb_n[a] + tau * nu * jtot[a];
            if (both) cv -= avgt_n[a];
            Cs[(a * 4 + 0) * L.FP + pt] = dA * cv;
            // physical coefficient of grad v_a: nu/2 (jadj_a n + n_a jadj), mapped to reference derivatives
            T pv[3], cf[3];
            for (int e = 0; e < 3; ++e) pv[e] = T(0.5) * nu * (jadj[a] * nv[e] + nv[a] * jadj[e]);
            phys_to_ref(Js, pv, cf);
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) Cs[(a * 4 + 1 + jj) * L.FP + pt] = dA * cf[ax[jj]];
            if (enr_c) {
              T cve = tau * nu * jtot[a];
              if (both) cve -= avgt_n[a];
              if (iface) cve -= avgb_n[a];
              Es[(a * 4 + 0) * L.FP + pt] = dA * cve;
              for (int b = 0; b < 3; ++b) {
                const T coef = both ? wt_s * (nu + nut_s) * (jtot[a] * nv[b] + nv[a] * jtot[b]) : T(0);
                Es[(a * 4 + 1 + b) * L.FP + pt] = dA * coef;
              }
            }
          }
        }
      }
    }
    __syncthreads();
    // enriched tests on these two faces
    if (enr_c && (OP == OP_CONV || OP == OP_VISC)) {
      auto contrib = [&](int t, T *acc, auto nvc) {
        constexpr int NV = decltype(nvc)::value;
        const int s = t / FP, pt = t - s * FP;
        const int a1 = pt % p1, a2 = pt / p1;
        T xs[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) xs[e] = e == d ? T(s) : (e == t1 ? B.x[s1][a1] : B.x[s2][a2]);
        const T f[3][2] = {{T(1) - xs[0], xs[0]}, {T(1) - xs[1], xs[1]}, {T(1) - xs[2], xs[2]}};
        const T *w = m.wt_face[opc] + (((size_t)ec * 6 + 2 * d + s) * m.fpmax[opc]) * WT + pt * WT;
        const T *Es = E + s * 3 * 4 * L.FP;
        T Js[3][3], dets;
        if (CURVED && OP == OP_VISC) load_rec(face_rec(m, B, col, d, s, s1, s2, a1, a2), Js, dets);
        T cv[3], cg[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          cv[a] = Es[(a * 4) * L.FP + pt] * w[0];
#pragma unroll
          for (int b = 0; b < 3; ++b) cg[a][b] = OP == OP_VISC ? Es[(a * 4 + 1 + b) * L.FP + pt] : T(0);
        }
        // value test psi N_v: beta_a = cv_a (+ cg_a . grad psi); gradient test grad(psi N_v):
        // alpha_a[e] = psi (J^-1 cg_a)_e
        T beta[3], alpha[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          beta[a] = cv[a];
#pragma unroll
          for (int e = 0; e < 3; ++e) alpha[a][e] = T(0);
          if (OP == OP_VISC) {
            beta[a] += cg[a][0] * w[1] + cg[a][1] * w[2] + cg[a][2] * w[3];
            if (NV == 8) {
              if (CURVED) {
                phys_to_ref(Js, cg[a], alpha[a]);
#pragma unroll
                for (int e = 0; e < 3; ++e) alpha[a][e] *= w[0];
              } else {
#pragma unroll
                for (int e = 0; e < 3; ++e) alpha[a][e] = w[0] * cg[a][e] * hinv[e];
              }
            }
          }
        }
        if (NV == 1) {
#pragma unroll
          for (int a = 0; a < 3; ++a) acc[a] += beta[a];
        } else {
          acc_trilinear<T>(f, beta, alpha, acc);
        }
      };
      reduce_enr<T>(l0, 2 * FP, contrib, re, S0 + L.part);
    }
    // I1: along t2 (p2 -> n); I2: along t1 (p1 -> n); item k = (face s, component a)
    T *I0 = S0 + L.fI0, *I1 = S0 + L.fI1, *I2 = S0 + L.fI2, *F2 = S0 + L.fF2, *G2 = S0 + L.fG2;
    const int ni = 2 * NOUT;
    pass_batch<T>([&](int b) -> Pass<T> {
      const int k = b % ni, j = b / ni;   // j: 0 I0 = S2^T f + D2^T ht2, 1 I1 = S2^T ht1, 2 I2 = S2^T hd
      const int s = k / NOUT, a = k % NOUT;
      const T *Ck = C + (s * 3 + a) * 4 * L.FP;
      if (j == 0) return {Ck, B.S[s2], GRAD ? Ck + 3 * L.FP : nullptr, B.D[s2], I0 + k * L.pn};
      if (j == 1) return {Ck + 2 * L.FP, B.S[s2], nullptr, nullptr, I1 + k * L.pn};
      return {Ck + 1 * L.FP, B.S[s2], nullptr, nullptr, I2 + k * L.pn};
    }, GRAD ? 3 * ni : ni, p1, p2, 1, 1, n, p2, true, false);
    pass_batch<T>([&](int b) -> Pass<T> {
      const int k = b % ni, j = b / ni;   // j: 0 F2 = S1^T I0 + D1^T I1, 1 G2 = S1^T I2
      if (j == 0) return {I0 + k * L.pn, B.S[s1], GRAD ? I1 + k * L.pn : nullptr, B.D[s1], F2 + k * nn};
      return {I2 + k * L.pn, B.S[s1], nullptr, nullptr, G2 + k * nn};
    }, GRAD ? 2 * ni : ni, p1, n, 1, 0, n, p1, true, false);
    // scatter the face-layer values and the normal-derivative coefficients into the cell nodes
    for (int t = threadIdx.x; t < NOUT * n3; t += blockDim.x) {
      const int a = t / n3, node = t - a * n3;
      const int id[3] = {node % n, (node / n) % n, node / nn};
      const int fi = id[t1] + n * id[t2];
      T add = T(0);
      for (int s = 0; s < 2; ++s) {
        const int k = s * NOUT + a;
        if (id[d] == (s ? n - 1 : 0)) add += F2[k * nn + fi];
        if (GRAD) add += B.dend[s][id[d]] * G2[k * nn + fi];
      }
      r[t] += add;
    }
    __syncthreads();
    }   // face groups
  }
  }
  // ================= store =================
  if (OP == OP_LAP && epi.mode != LAP_PLAIN) {
    const size_t o = (size_t)c * n3;
    for (int t = threadIdx.x; t < n3; t += blockDim.x) {
      const size_t i = o + t;
      if (epi.mode == LAP_RESIDUAL) {
        y[i] = epi.b[i] - r[t];
      } else {
        const T dn = (epi.first ? T(0) : epi.c1 * epi.d[i]) + epi.c2 * epi.dinv[i] * (epi.b[i] - r[t]);
        epi.d[i] = dn;
        epi.xout[i] = u[i] + dn;
      }
    }
  } else if (NOUT == 1) {
    T *yc = y + (size_t)c * n3;
    for (int t = threadIdx.x; t < n3; t += blockDim.x) yc[t] = r[t];
  } else {
    T *yc = y + (size_t)c * 3 * n3;
    for (int t = threadIdx.x; t < 3 * n3; t += blockDim.x) yc[t] = r[t];
    if (!enr_c && m.slot && m.slot[c] >= 0) {
      // wall model switched off in this cell: its enrichment coefficients have no function
      for (int t = threadIdx.x; t < 3 * m.nef; t += blockDim.x) y[3 * m.np + (size_t)m.slot[c] * 3 * m.nef + t] = T(0);
    } else if (enr_c && m.nef == 8)
      for (int t = threadIdx.x; t < 24; t += blockDim.x) y[3 * m.np + (size_t)ec * 24 + t] = re[t];
    else if (enr_c && threadIdx.x < 3)   // l = 0: the integrals of psi e_a, accumulated in re[a]
      y[3 * m.np + (size_t)ec * 3 + threadIdx.x] = re[threadIdx.x];
  }
}

// rows [0, rb) and [rt, ny) (default: every row)
template <typename T, int OP, int GEO, int NC = 0>
static cudaError_t launch_vec(const MeshView<T> &m, const T *u, T *y, cudaStream_t s, const LapEpi<T> *epi, int rb = -1,
                              int rt = -1) {
  if (rb < 0) rb = rt = m.ny;
  const int nr = rb + (m.ny - rt);
  if (nr <= 0) return cudaSuccess;
  const int qset = OP == OP_CONV ? QSET_CONV : QSET_LIN;
  const VecPlan L = vec_plan(OP, GEO == GEO_CURVED, m.n1, plan_qin(m, qset), m.q[QSET_WALL]);
  const size_t sm = ((sizeof(Basis<T>) + 15) / 16) * 16 + (size_t)L.total * sizeof(T);
  if (sm > 220 * 1024) return cudaErrorInvalidConfiguration;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(vector_op_kernel<T, OP, GEO, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         220 * 1024);
    if (e == cudaSuccess)   // the whole unified L1/shared array as shared memory: more CTAs per SM
      e = cudaFuncSetAttribute(vector_op_kernel<T, OP, GEO, NC>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  note_launch();
  LapEpi<T> e{};
  e.mode = LAP_PLAIN;
  if (epi) e = *epi;
  vector_op_kernel<T, OP, GEO, NC><<<m.nx * nr * m.nz, 128, sm, s>>>(m, u, y, e, rb, rt);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vector_op(int op, const MeshView<T> &m, const T *u, T *y, cudaStream_t s, const LapEpi<T> *epi) {
  note_dofs((op == OP_DIV || op == OP_LAP) ? m.np : m.nu);
  if (m.geo == GEO_BOX && (op == OP_DIV || op == OP_VISC || op == OP_CONV) && m.plain_hi > m.plain_lo) {
    // rows of standard cells: degree-specialised kernels; the rows of the enriched layers (and, with
    // the q_w^3 rule, the rows next to them): the general kernel
    cudaError_t e = launch_box_vec_rows<T, T>(op, m, u, y, m.plain_lo, m.plain_hi - m.plain_lo, s);
    if (e != cudaSuccess) return e;
    if (op == OP_DIV) return launch_vec<T, OP_DIV, GEO_BOX>(m, u, y, s, nullptr, m.plain_lo, m.plain_hi);
    if (op == OP_CONV) return launch_vec<T, OP_CONV, GEO_BOX>(m, u, y, s, nullptr, m.plain_lo, m.plain_hi);
    return launch_vec<T, OP_VISC, GEO_BOX>(m, u, y, s, nullptr, m.plain_lo, m.plain_hi);
  }
  if (m.geo == GEO_BOX && (op == OP_MASS || op == OP_DIVDIV) && m.std_hi > m.std_lo) {
    // volume-only operators: box kernels on every row without enrichment slots, the general kernel
    // on the wall layers
    cudaError_t e = launch_box_vec_rows<T, T>(op, m, u, y, m.std_lo, m.std_hi - m.std_lo, s);
    if (e != cudaSuccess) return e;
    if (op == OP_MASS) return launch_vec<T, OP_MASS, GEO_BOX>(m, u, y, s, nullptr, m.std_lo, m.std_hi);
    return launch_vec<T, OP_DIVDIV, GEO_BOX>(m, u, y, s, nullptr, m.std_lo, m.std_hi);
  }
  if (m.geo == GEO_CURVED) {
    switch (op) {
      case OP_DIV: return launch_vec<T, OP_DIV, GEO_CURVED>(m, u, y, s, nullptr);
      case OP_CONV: return launch_vec<T, OP_CONV, GEO_CURVED>(m, u, y, s, nullptr);
      case OP_VISC: return launch_vec<T, OP_VISC, GEO_CURVED>(m, u, y, s, nullptr);
      case OP_MASS: return launch_vec<T, OP_MASS, GEO_CURVED>(m, u, y, s, nullptr);
      case OP_DIVDIV: return launch_vec<T, OP_DIVDIV, GEO_CURVED>(m, u, y, s, nullptr);
      case OP_LAP:
        switch (m.n1) {
          case 2: return launch_vec<T, OP_LAP, GEO_CURVED, 2>(m, u, y, s, epi);
          case 3: return launch_vec<T, OP_LAP, GEO_CURVED, 3>(m, u, y, s, epi);
          case 4: return launch_vec<T, OP_LAP, GEO_CURVED, 4>(m, u, y, s, epi);
          case 5: return launch_vec<T, OP_LAP, GEO_CURVED, 5>(m, u, y, s, epi);
          case 6: return launch_vec<T, OP_LAP, GEO_CURVED, 6>(m, u, y, s, epi);
        }
        return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
  }
  switch (op) {
    case OP_DIV: return launch_vec<T, OP_DIV, GEO_BOX>(m, u, y, s, nullptr);
    case OP_CONV: return launch_vec<T, OP_CONV, GEO_BOX>(m, u, y, s, nullptr);
    case OP_VISC: return launch_vec<T, OP_VISC, GEO_BOX>(m, u, y, s, nullptr);
    case OP_MASS: return launch_vec<T, OP_MASS, GEO_BOX>(m, u, y, s, nullptr);
    case OP_DIVDIV: return launch_vec<T, OP_DIVDIV, GEO_BOX>(m, u, y, s, nullptr);
  }
  return cudaErrorInvalidValue;
}

template cudaError_t launch_vector_op<double>(int, const MeshView<double> &, const double *, double *, cudaStream_t,
                                              const LapEpi<double> *);

cudaError_t launch_cfl_rate(const MeshView<double> &m, const double *u, double *rate, cudaStream_t s) {
  if (m.geo == GEO_CURVED) return launch_vec<double, OP_CFL, GEO_CURVED>(m, u, rate, s, nullptr);
  return launch_vec<double, OP_CFL, GEO_BOX>(m, u, rate, s, nullptr);
}

cudaError_t launch_vector_op_df(int op, const MeshView<double> &m, const double *u, double *y, cudaStream_t s) {
  if (m.geo != GEO_BOX || (op != OP_DIV && op != OP_VISC && op != OP_CONV)) return cudaErrorNotSupported;
  note_dofs(op == OP_DIV ? m.np : m.nu);
  if (m.plain_hi > m.plain_lo) {
    cudaError_t e = launch_box_vec_rows<double, df64>(op, m, u, y, m.plain_lo, m.plain_hi - m.plain_lo, s);
    if (e != cudaSuccess) return e;
  }
  if (op == OP_DIV) return launch_vec<double, OP_DIV, GEO_BOX>(m, u, y, s, nullptr, m.plain_lo, m.plain_hi);
  if (op == OP_CONV) return launch_vec<double, OP_CONV, GEO_BOX>(m, u, y, s, nullptr, m.plain_lo, m.plain_hi);
  return launch_vec<double, OP_VISC, GEO_BOX>(m, u, y, s, nullptr, m.plain_lo, m.plain_hi);
}
template cudaError_t launch_vector_op<float>(int, const MeshView<float> &, const float *, float *, cudaStream_t,
                                             const LapEpi<float> *);

}  // namespace dgw
