// Matrix-free DG operator kernels on the channel of boxes (one CTA per cell, shared-memory
// sum factorisation; Sec. 4.4). Every CTA evaluates the volume integral of its cell and the
// integrals over its six faces for its own test functions, re-reading the neighbour's
// coefficients (cell-centric face loop: no atomics, deterministic).
//
//   vector_op_kernel : OP_DIV  b = -C(q,u)                   (Sec. 4.2, velocity divergence)
//                      OP_CONV y = F^c(v,u), LF flux          (Sec. 4.2, convective term)
//                      OP_VISC y = -F^nu(vbar,v~;ubar,u~)     (eq. viscous_multiscale)
// Wall-layer cells add the enrichment u~ = psi sum_B N_B u~_B (eq. enrichment) at q_wall
// wall-normal Gauss points, with psi and grad psi read from the wall tables.
#include "sumfac.cuh"

namespace dgw {

template <typename T>
__device__ __forceinline__ void cell_ijk(const MeshView<T> &m, int c, int &i, int &j, int &kz) {
  i = c % m.nx;
  j = (c / m.nx) % m.ny;
  kz = c / (m.nx * m.ny);
}

// neighbour across face f = 2d + side, -1 on a wall
template <typename T>
__device__ __forceinline__ int neighbour(const MeshView<T> &m, int c, int f) {
  int i, j, kz;
  cell_ijk(m, c, i, j, kz);
  const int d = f >> 1, s = (f & 1) ? 1 : -1;
  if (d == 0) i = (i + s + m.nx) % m.nx;
  else if (d == 2) kz = (kz + s + m.nz) % m.nz;
  else {
    j += s;
    if (j < 0 || j >= m.ny) return -1;
  }
  return i + m.nx * (j + m.ny * kz);
}

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

// ------------------------------------------------------------------------------------------
// Vector operators (divergence, convective, viscous) with enriched wall cells
// ------------------------------------------------------------------------------------------

struct VecLayout {
  int n, n3, P, FP, tsz;
  // offsets in T words
  int uo, un, r, eo, en, re, vol, face, tmp, total;
};

__host__ __device__ inline VecLayout vec_layout(int op, int n, int qin, int qw) {
  VecLayout L;
  L.n = n;
  L.n3 = n * n * n;
  const int qy = qw > qin ? qw : qin;
  L.P = qin * qy * qin;
  L.FP = qin * qy;
  const int qm = qy > n ? qy : n;
  int a = qin * n * n, b = qin * qy * n, c = n * (n > qm ? n : qm);
  L.tsz = 5 * (a > b ? (a > c ? a : c) : (b > c ? b : c));
  int o = 0;
  L.uo = o; o += 3 * L.n3;
  L.un = o; o += 3 * L.n3;
  L.r = o; o += 3 * L.n3;
  L.eo = o; o += 24;
  L.en = o; o += 24;
  L.re = o; o += 24;
  L.vol = o;
  // volume arrays: DIV 3 (U) + 3 (H); CONV 3 (U) + 9 (H); VISC 9 (Gb/H) + 9 (Gt)
  o += (op == OP_DIV ? 6 : (op == OP_CONV ? 12 : 18)) * L.P;
  L.face = o;
  // face arrays: per side 3 values + 9 gradients (VISC) or 3 values; coefficients 12 + enriched 12
  o += (op == OP_VISC ? (2 * 12 + 12 + 12) : (2 * 3 + 4 + 3)) * L.FP;
  L.tmp = o;
  o += L.tsz;
  L.total = o;
  return L;
}

template <typename T, int OP>
__global__ void __launch_bounds__(128) vector_op_kernel(MeshView<T> m, const T *__restrict__ u, T *__restrict__ y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Basis<T> &B = *reinterpret_cast<Basis<T> *>(smem_raw);
  T *S0 = reinterpret_cast<T *>(smem_raw + ((sizeof(Basis<T>) + 15) / 16) * 16);
  load_basis(m.basis, &B);
  __syncthreads();
  const int n = m.n1;
  const int qset = OP == OP_CONV ? QSET_CONV : QSET_LIN;
  const int opc = OP == OP_CONV ? 1 : 0;   // wall-table class
  const int qin = B.q[qset], qw = B.q[QSET_WALL];
  const VecLayout L = vec_layout(OP, n, qin, qw);
  const int n3 = L.n3;
  T *uo = S0 + L.uo, *un = S0 + L.un, *r = S0 + L.r, *eo = S0 + L.eo, *en = S0 + L.en, *re = S0 + L.re;
  T *tmp = S0 + L.tmp;
  const int c = blockIdx.x;
  const int ec = m.enr[c];
  const bool enr_c = ec >= 0;
  const int ncomp_out = OP == OP_DIV ? 1 : 3;
  const T nu = m.visc;
  // load own coefficients
  for (int t = threadIdx.x; t < 3 * n3; t += blockDim.x) {
    uo[t] = u[(size_t)c * 3 * n3 + t];
    r[t] = T(0);
  }
  if (enr_c)
    for (int t = threadIdx.x; t < 24; t += blockDim.x) { eo[t] = u[3 * m.np + (size_t)ec * 24 + t]; re[t] = T(0); }
  __syncthreads();
  const T h[3] = {m.hx, m.hy[(c / m.nx) % m.ny], m.hz};
  const T hinv[3] = {T(1) / h[0], T(1) / h[1], T(1) / h[2]};
  const int ys = enr_c ? QSET_WALL : qset;
  AxisTabs<T> tabs;
  const int sets[3] = {qset, ys, qset};
  for (int d = 0; d < 3; ++d) { tabs.S[d] = B.S[sets[d]]; tabs.D[d] = B.D[sets[d]]; tabs.q[d] = B.q[sets[d]]; }
  const int q0 = tabs.q[0], q1 = tabs.q[1], q2 = tabs.q[2];
  const int P = q0 * q1 * q2;
  const T vol = h[0] * h[1] * h[2];
  const T *wtv = enr_c ? m.wt_vol[opc] + (size_t)ec * m.nvol[opc] * WT : nullptr;

  // ---------------- volume ----------------
  T *V = S0 + L.vol;
  if (OP == OP_DIV || OP == OP_CONV) {
    T *U = V;            // 3 x P values
    T *H = V + 3 * L.P;  // DIV: 3 x P ; CONV: 9 x P
    for (int a = 0; a < 3; ++a) eval_cell(uo + a * n3, n, tabs, U + a * L.P, (T *)nullptr, (T *)nullptr, (T *)nullptr, tmp);
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
      const int i0 = t % q0, i1 = (t / q0) % q1, i2 = t / (q0 * q1);
      T uu[3] = {U[t], U[L.P + t], U[2 * L.P + t]};
      if (enr_c) {
        const T xi[3] = {B.x[sets[0]][i0], B.x[sets[1]][i1], B.x[sets[2]][i2]};
        T N[8], dN[8][3];
        q1_weights(xi, N, dN);
        const T psi = wtv[t * WT];
        for (int a = 0; a < 3; ++a) {
          T s = T(0);
          for (int v = 0; v < 8; ++v) s += N[v] * eo[a * 8 + v];
          uu[a] += psi * s;
          U[a * L.P + t] = uu[a];
        }
      }
      const T dV = vol * B.w[sets[0]][i0] * B.w[sets[1]][i1] * B.w[sets[2]][i2];
      if (OP == OP_DIV) {
        for (int d = 0; d < 3; ++d) H[d * L.P + t] = dV * uu[d] * hinv[d];
      } else {
        for (int a = 0; a < 3; ++a)
          for (int d = 0; d < 3; ++d) H[(a * 3 + d) * L.P + t] = -dV * uu[a] * uu[d] * hinv[d];
      }
    }
    __syncthreads();
    if (OP == OP_DIV) {
      integrate_cell((const T *)nullptr, H, H + L.P, H + 2 * L.P, n, tabs, r, tmp);
    } else {
      for (int a = 0; a < 3; ++a)
        integrate_cell((const T *)nullptr, H + (a * 3) * L.P, H + (a * 3 + 1) * L.P, H + (a * 3 + 2) * L.P, n, tabs,
                       r + a * n3, tmp);
      if (enr_c) {
        // enriched tests: -(grad(psi N_v) e_a, u x u)
        auto val = [&](int o, int t) -> T {
          const int a = o >> 3, v = o & 7;
          const int i0 = t % q0, i1 = (t / q0) % q1, i2 = t / (q0 * q1);
          const T xi[3] = {B.x[sets[0]][i0], B.x[sets[1]][i1], B.x[sets[2]][i2]};
          T N[8], dN[8][3];
          q1_weights(xi, N, dN);
          const T *w = wtv + t * WT;
          T ug = T(0);
          for (int d = 0; d < 3; ++d) ug += U[d * L.P + t] * (w[0] * dN[v][d] * hinv[d] + N[v] * w[1 + d]);
          const T dV = vol * B.w[sets[0]][i0] * B.w[sets[1]][i1] * B.w[sets[2]][i2];
          return -dV * U[a * L.P + t] * ug;
        };
        reduce_outputs(24, P, val, re);
      }
    }
  } else {  // OP_VISC
    T *G = V;             // 9 x P: grad ubar (then test coefficients)
    T *Gt = V + 9 * L.P;  // 9 x P: grad u~ (physical)
    for (int a = 0; a < 3; ++a)
      eval_cell(uo + a * n3, n, tabs, (T *)nullptr, G + (a * 3) * L.P, G + (a * 3 + 1) * L.P, G + (a * 3 + 2) * L.P, tmp);
    const T *nutv = enr_c ? m.nut_vol + (size_t)ec * m.nvol[0] : nullptr;
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
      const int i0 = t % q0, i1 = (t / q0) % q1, i2 = t / (q0 * q1);
      T gb[3][3], tb[3][3];
      for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) gb[a][d] = G[(a * 3 + d) * L.P + t] * hinv[d];
      for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) tb[a][d] = nu * (gb[a][d] + gb[d][a]);
      if (enr_c) {
        const T xi[3] = {B.x[sets[0]][i0], B.x[sets[1]][i1], B.x[sets[2]][i2]};
        T N[8], dN[8][3];
        q1_weights(xi, N, dN);
        const T *w = wtv + t * WT;
        T gt[3][3];
        for (int a = 0; a < 3; ++a)
          for (int d = 0; d < 3; ++d) {
            T s = T(0);
            for (int v = 0; v < 8; ++v) s += eo[a * 8 + v] * (w[0] * dN[v][d] * hinv[d] + N[v] * w[1 + d]);
            gt[a][d] = s;
            Gt[(a * 3 + d) * L.P + t] = s;
          }
        const T nut = nutv[t];
        const T nuh = min(nu + nut, T(2) * sqrt(nu * (nu + nut)));   // eq. (minvt)
        for (int a = 0; a < 3; ++a)
          for (int d = 0; d < 3; ++d) tb[a][d] += nuh * (gt[a][d] + gt[d][a]);
      }
      const T dV = vol * B.w[sets[0]][i0] * B.w[sets[1]][i1] * B.w[sets[2]][i2];
      for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) G[(a * 3 + d) * L.P + t] = dV * tb[a][d] * hinv[d];
    }
    __syncthreads();
    for (int a = 0; a < 3; ++a)
      integrate_cell((const T *)nullptr, G + (a * 3) * L.P, G + (a * 3 + 1) * L.P, G + (a * 3 + 2) * L.P, n, tabs,
                     r + a * n3, tmp);
    if (enr_c) {
      // enriched tests: (eps(psi N_v e_a), 2(nu+nu_t) eps(u~))
      auto val = [&](int o, int t) -> T {
        const int a = o >> 3, v = o & 7;
        const int i0 = t % q0, i1 = (t / q0) % q1, i2 = t / (q0 * q1);
        const T xi[3] = {B.x[sets[0]][i0], B.x[sets[1]][i1], B.x[sets[2]][i2]};
        T N[8], dN[8][3];
        q1_weights(xi, N, dN);
        const T *w = wtv + t * WT;
        const T nut = nutv[t];
        T s = T(0);
        for (int d = 0; d < 3; ++d) {
          const T gv = w[0] * dN[v][d] * hinv[d] + N[v] * w[1 + d];
          s += gv * (nu + nut) * (Gt[(a * 3 + d) * L.P + t] + Gt[(d * 3 + a) * L.P + t]);
        }
        const T dV = vol * B.w[sets[0]][i0] * B.w[sets[1]][i1] * B.w[sets[2]][i2];
        return dV * s;
      };
      reduce_outputs(24, P, val, re);
    }
  }

  // ---------------- faces ----------------
  T *F = S0 + L.face;
  for (int f = 0; f < 6; ++f) {
    const int nb = neighbour(m, c, f);
    const int d = f >> 1, side = f & 1;
    int t1, t2;
    face_axes(d, t1, t2);
    const int eb = nb >= 0 ? m.enr[nb] : -1;
    const bool enr_o = nb >= 0 ? eb >= 0 : enr_c;
    const bool both = enr_c && enr_o, iface = enr_c != enr_o;
    const int s1 = (t1 == 1 && (enr_c || enr_o)) ? QSET_WALL : qset;
    const int s2 = (t2 == 1 && (enr_c || enr_o)) ? QSET_WALL : qset;
    const int p1 = B.q[s1], p2 = B.q[s2], FP = p1 * p2;
    if (nb >= 0) {
      for (int t = threadIdx.x; t < 3 * n3; t += blockDim.x) un[t] = u[(size_t)nb * 3 * n3 + t];
      if (eb >= 0)
        for (int t = threadIdx.x; t < 24; t += blockDim.x) en[t] = u[3 * m.np + (size_t)eb * 24 + t];
      __syncthreads();
    }
    const T sgn = side ? T(1) : T(-1);
    const T hd = h[d];
    const T hdo = nb >= 0 ? cell_h(m, nb, d) : hd;
    const T area = h[t1] * h[t2];
    const T *wts = enr_c ? m.wt_face[opc] + (((size_t)ec * 6 + f) * m.fpmax[opc]) * WT : nullptr;
    const T *wto = (nb >= 0 && eb >= 0) ? m.wt_face[opc] + (((size_t)eb * 6 + (f ^ 1)) * m.fpmax[opc]) * WT : nullptr;
    // traces: own values Vs[3], neighbour Vo[3]; VISC: gradients (reference d, t1, t2)
    T *Vs = F, *Vo = F + 3 * L.FP;
    T *Gs = nullptr, *Go = nullptr, *C = nullptr, *E = nullptr;
    if (OP == OP_VISC) {
      Gs = F + 6 * L.FP;       // 9: [a][dir d,t1,t2]
      Go = F + 15 * L.FP;      // 9
      C = F + 24 * L.FP;       // 12: per component f, hd, ht1, ht2
      E = F + 36 * L.FP;       // 12: per component value coeff + 3 physical gradient coeffs (enriched tests)
    } else {
      C = F + 6 * L.FP;        // DIV: 1 (f) ; CONV: 3 (f per component)
      E = F + 10 * L.FP;       // CONV enriched value coeffs (3)
    }
    const T *S1 = B.S[s1], *D1 = B.D[s1], *Sb2 = B.S[s2], *D2 = B.D[s2];
    for (int a = 0; a < 3; ++a) {
      if (OP == OP_VISC)
        eval_face(uo + a * n3, n, d, side, B.dend[side], S1, D1, p1, Sb2, D2, p2, Vs + a * L.FP, Gs + (a * 3) * L.FP,
                  Gs + (a * 3 + 1) * L.FP, Gs + (a * 3 + 2) * L.FP, tmp);
      else
        eval_face(uo + a * n3, n, d, side, B.dend[side], S1, D1, p1, Sb2, D2, p2, Vs + a * L.FP, (T *)nullptr,
                  (T *)nullptr, (T *)nullptr, tmp);
      if (nb >= 0) {
        if (OP == OP_VISC)
          eval_face(un + a * n3, n, d, 1 - side, B.dend[1 - side], S1, D1, p1, Sb2, D2, p2, Vo + a * L.FP,
                    Go + (a * 3) * L.FP, Go + (a * 3 + 1) * L.FP, Go + (a * 3 + 2) * L.FP, tmp);
        else
          eval_face(un + a * n3, n, d, 1 - side, B.dend[1 - side], S1, D1, p1, Sb2, D2, p2, Vo + a * L.FP,
                    (T *)nullptr, (T *)nullptr, (T *)nullptr, tmp);
      }
    }
    const T tau = nb >= 0 ? max(m.tau[c], m.tau[nb]) : T(10) * m.tau[c];
    const T *nuts = (OP == OP_VISC && enr_c) ? m.nut_face + ((size_t)ec * 6 + f) * m.fpmax[0] : nullptr;
    const T *nuto = (OP == OP_VISC && nb >= 0 && eb >= 0) ? m.nut_face + ((size_t)eb * 6 + (f ^ 1)) * m.fpmax[0] : nullptr;
    for (int t = threadIdx.x; t < FP; t += blockDim.x) {
      const int a1 = t % p1, a2 = t / p1;
      const T dA = area * B.w[s1][a1] * B.w[s2][a2];
      // physical point coordinates on both sides
      T xs[3], xo[3];
      xs[d] = T(side); xs[t1] = B.x[s1][a1]; xs[t2] = B.x[s2][a2];
      xo[d] = T(1 - side); xo[t1] = xs[t1]; xo[t2] = xs[t2];
      T ub_s[3], ub_o[3], ut_s[3] = {0, 0, 0}, ut_o[3] = {0, 0, 0};
      T gbs[3][3], gbo[3][3], gts[3][3], gto[3][3];
      T Ns[8], dNs[8][3], No[8], dNo[8][3];
      if (enr_c) q1_weights(xs, Ns, dNs);
      if (nb >= 0 && eb >= 0) q1_weights(xo, No, dNo);
      for (int a = 0; a < 3; ++a) {
        ub_s[a] = Vs[a * L.FP + t];
        if (OP == OP_VISC) {
          T gref[3] = {Gs[(a * 3) * L.FP + t], Gs[(a * 3 + 1) * L.FP + t], Gs[(a * 3 + 2) * L.FP + t]};
          gbs[a][d] = gref[0] * hinv[d]; gbs[a][t1] = gref[1] * hinv[t1]; gbs[a][t2] = gref[2] * hinv[t2];
        }
        if (enr_c) {
          const T *w = wts + t * WT;
          T s = T(0);
          for (int v = 0; v < 8; ++v) s += Ns[v] * eo[a * 8 + v];
          ut_s[a] = w[0] * s;
          if (OP == OP_VISC)
            for (int e = 0; e < 3; ++e) {
              T g = T(0);
              for (int v = 0; v < 8; ++v) g += eo[a * 8 + v] * (w[0] * dNs[v][e] * hinv[e] + Ns[v] * w[1 + e]);
              gts[a][e] = g;
            }
        } else if (OP == OP_VISC) {
          gts[a][0] = gts[a][1] = gts[a][2] = T(0);
        }
        if (nb >= 0) {
          ub_o[a] = Vo[a * L.FP + t];
          if (OP == OP_VISC) {
            T gref[3] = {Go[(a * 3) * L.FP + t], Go[(a * 3 + 1) * L.FP + t], Go[(a * 3 + 2) * L.FP + t]};
            const T hto1 = (t1 == 1) ? cell_h(m, nb, 1) : h[t1];
            const T hto2 = (t2 == 1) ? cell_h(m, nb, 1) : h[t2];
            gbo[a][d] = gref[0] / hdo; gbo[a][t1] = gref[1] / hto1; gbo[a][t2] = gref[2] / hto2;
          }
          if (eb >= 0) {
            const T *w = wto + t * WT;
            T s = T(0);
            for (int v = 0; v < 8; ++v) s += No[v] * en[a * 8 + v];
            ut_o[a] = w[0] * s;
            if (OP == OP_VISC) {
              const T hob[3] = {m.hx, cell_h(m, nb, 1), m.hz};
              for (int e = 0; e < 3; ++e) {
                T g = T(0);
                for (int v = 0; v < 8; ++v) g += en[a * 8 + v] * (w[0] * dNo[v][e] / hob[e] + No[v] * w[1 + e]);
                gto[a][e] = g;
              }
            }
          } else if (OP == OP_VISC) {
            gto[a][0] = gto[a][1] = gto[a][2] = T(0);
          }
        } else {
          // mirror principle on no-slip walls: u+ = -u-, grad u+ = grad u-
          ub_o[a] = -ub_s[a];
          ut_o[a] = -ut_s[a];
          if (OP == OP_VISC)
            for (int e = 0; e < 3; ++e) { gbo[a][e] = gbs[a][e]; gto[a][e] = gts[a][e]; }
        }
      }
      if (OP == OP_DIV) {
        // -(q, {{u}}.n), wall: u^-
        const T us = ub_s[d] + ut_s[d], uo_ = ub_o[d] + ut_o[d];
        const T avg = nb >= 0 ? T(0.5) * (us + uo_) : us;
        C[t] = -dA * sgn * avg;
      } else if (OP == OP_CONV) {
        T um[3], up[3];
        for (int a = 0; a < 3; ++a) { um[a] = ub_s[a] + ut_s[a]; up[a] = ub_o[a] + ut_o[a]; }
        const T unm = sgn * um[d], unp = sgn * up[d];
        const T lam = max(T(2) * fabs(unm), T(2) * fabs(unp));
        for (int a = 0; a < 3; ++a) {
          const T Fa = T(0.5) * (um[a] * unm + up[a] * unp) + T(0.5) * lam * (um[a] - up[a]);
          C[a * L.FP + t] = dA * Fa;
          E[a * L.FP + t] = dA * Fa;
        }
      } else {  // VISC
        const T nut_s = nuts ? nuts[t] : T(0);
        const T nut_o = nb >= 0 ? (nuto ? nuto[t] : T(0)) : nut_s;
        T jb[3], jt[3], jtot[3], avgb_n[3], avgt_n[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) {
          jb[a] = ub_s[a] - ub_o[a];
          jt[a] = ut_s[a] - ut_o[a];
          jtot[a] = jb[a] + jt[a];
          // {{F^nu(ubar)}}.n with n = sgn e_d
          avgb_n[a] = T(0.5) * nu * sgn * ((gbs[a][d] + gbs[d][a]) + (gbo[a][d] + gbo[d][a]));
        }
        T wt_s = T(0.5);
        if (both) {
          const T den = T(2) * nu + nut_s + nut_o;
          wt_s = (nu + nut_o) / den;
          const T wt_o = (nu + nut_s) / den;
          for (int a = 0; a < 3; ++a)
            avgt_n[a] = sgn * (wt_s * (nu + nut_s) * (gts[a][d] + gts[d][a]) + wt_o * (nu + nut_o) * (gto[a][d] + gto[d][a]));
        }
        T jadj[3];
        for (int a = 0; a < 3; ++a) jadj[a] = jb[a] + (iface ? jt[a] : T(0));
        for (int a = 0; a < 3; ++a) {
          T cv = -avgb_n[a] + tau * nu * jtot[a];
          if (both) cv -= avgt_n[a];
          // coefficient of phi: dA cv; of dphi/dxi_b: dA nu/2 sgn (jadj_a delta_bd + delta_ad jadj_b)/h_b
          C[(a * 4 + 0) * L.FP + t] = dA * cv;
          C[(a * 4 + 1) * L.FP + t] = dA * T(0.5) * nu * sgn * (jadj[a] + (a == d ? jadj[d] : T(0))) * hinv[d];
          C[(a * 4 + 2) * L.FP + t] = dA * T(0.5) * nu * sgn * (a == d ? jadj[t1] : T(0)) * hinv[t1];
          C[(a * 4 + 3) * L.FP + t] = dA * T(0.5) * nu * sgn * (a == d ? jadj[t2] : T(0)) * hinv[t2];
          if (enr_c) {
            T cve = tau * nu * jtot[a];
            if (both) cve -= avgt_n[a];
            if (iface) cve -= avgb_n[a];
            E[(a * 4 + 0) * L.FP + t] = dA * cve;
            for (int b = 0; b < 3; ++b) {
              // (w F^{nu+nut}(v~), [[u~]] + [[ubar]]) on d Omega~_e: physical-gradient coefficient
              const T coef = both ? wt_s * (nu + nut_s) * sgn * ((b == d ? jtot[a] : T(0)) + (a == d ? jtot[b] : T(0))) : T(0);
              E[(a * 4 + 1 + b) * L.FP + t] = dA * coef;
            }
          }
        }
      }
    }
    __syncthreads();
    if (OP == OP_DIV) {
      integrate_face(C, (const T *)nullptr, (const T *)nullptr, (const T *)nullptr, n, d, side, B.dend[side], S1, D1,
                     p1, Sb2, D2, p2, r, tmp);
    } else if (OP == OP_CONV) {
      for (int a = 0; a < 3; ++a)
        integrate_face(C + a * L.FP, (const T *)nullptr, (const T *)nullptr, (const T *)nullptr, n, d, side,
                       B.dend[side], S1, D1, p1, Sb2, D2, p2, r + a * n3, tmp);
      if (enr_c) {
        auto val = [&](int o, int t) -> T {
          const int a = o >> 3, v = o & 7;
          const int a1 = t % p1, a2 = t / p1;
          T xs[3];
          xs[d] = T(side); xs[t1] = B.x[s1][a1]; xs[t2] = B.x[s2][a2];
          T N[8], dN[8][3];
          q1_weights(xs, N, dN);
          return E[a * L.FP + t] * wts[t * WT] * N[v];
        };
        reduce_outputs(24, FP, val, re);
      }
    } else {
      for (int a = 0; a < 3; ++a)
        integrate_face(C + (a * 4) * L.FP, C + (a * 4 + 1) * L.FP, C + (a * 4 + 2) * L.FP, C + (a * 4 + 3) * L.FP, n, d,
                       side, B.dend[side], S1, D1, p1, Sb2, D2, p2, r + a * n3, tmp);
      if (enr_c) {
        auto val = [&](int o, int t) -> T {
          const int a = o >> 3, v = o & 7;
          const int a1 = t % p1, a2 = t / p1;
          T xs[3];
          xs[d] = T(side); xs[t1] = B.x[s1][a1]; xs[t2] = B.x[s2][a2];
          T N[8], dN[8][3];
          q1_weights(xs, N, dN);
          const T *w = wts + t * WT;
          T s = E[(a * 4) * L.FP + t] * w[0] * N[v];
          for (int b = 0; b < 3; ++b) s += E[(a * 4 + 1 + b) * L.FP + t] * (w[0] * dN[v][b] * hinv[b] + N[v] * w[1 + b]);
          return s;
        };
        reduce_outputs(24, FP, val, re);
      }
    }
  }
  // ---------------- store ----------------
  if (OP == OP_DIV) {
    T *yc = y + (size_t)c * n3;
    for (int t = threadIdx.x; t < n3; t += blockDim.x) yc[t] = r[t];
  } else {
    T *yc = y + (size_t)c * 3 * n3;
    for (int t = threadIdx.x; t < 3 * n3; t += blockDim.x) yc[t] = r[t];
    if (enr_c)
      for (int t = threadIdx.x; t < 24; t += blockDim.x) y[3 * m.np + (size_t)ec * 24 + t] = re[t];
  }
  (void)ncomp_out;
}

template <typename T, int OP>
static cudaError_t launch_vec(const MeshView<T> &m, const T *u, T *y, cudaStream_t s) {
  const int qset = OP == OP_CONV ? QSET_CONV : QSET_LIN;
  const VecLayout L = vec_layout(OP, m.n1, m.q[qset], m.q[QSET_WALL]);
  const size_t sm = ((sizeof(Basis<T>) + 15) / 16) * 16 + (size_t)L.total * sizeof(T);
  if (sm > 220 * 1024) return cudaErrorInvalidConfiguration;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(vector_op_kernel<T, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  note_launch();
  note_dofs(OP == OP_DIV ? m.np : m.nu);
  vector_op_kernel<T, OP><<<m.nc, 128, sm, s>>>(m, u, y);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vector_op(int op, const MeshView<T> &m, const T *u, T *y, cudaStream_t s) {
  switch (op) {
    case OP_DIV: return launch_vec<T, OP_DIV>(m, u, y, s);
    case OP_CONV: return launch_vec<T, OP_CONV>(m, u, y, s);
    case OP_VISC: return launch_vec<T, OP_VISC>(m, u, y, s);
  }
  return cudaErrorInvalidValue;
}

template cudaError_t launch_vector_op<double>(int, const MeshView<double> &, const double *, double *, cudaStream_t);
template cudaError_t launch_vector_op<float>(int, const MeshView<float> &, const float *, float *, cudaStream_t);

}  // namespace dgw
