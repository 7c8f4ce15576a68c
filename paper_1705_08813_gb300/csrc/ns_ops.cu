// Operators of the projection step of the dual-splitting scheme (Sec. 4.2, eq. projectionspat):
//   NS_GRAD   y = P(v, p) = -(div v, p)_K + (v, {{p}} n)_dK, {{p}} = p^- on walls
//   NS_TAU    tau_D = |u|_K h dt / Cr per cell (eq. tauD), |u|_K the volume average, h = vol^(1/3)
//   NS_CURL   y = (v, curl u)_K, the right-hand side of the vorticity's L2 projection (Sec. 4.2)
// One CTA per cell with shared-memory sum factorisation over the cell's velocity point set (k+1
// Gauss points, q_w wall-normal in cells with the wall model switched on); enriched test
// functions psi N_v e_a through the wall tables. The gradient maps a scalar per point, f(t), to the
// test functions' divergences: the coefficient of d phi / d xi_d in output component a is
// f J^-1[d][a]. (The div-div penalty of the same step runs in the general operator kernel.)
#include <cmath>

#include "dgw_internal.h"
#include "metric.cuh"
#include "sumfac.cuh"

namespace dgw {

namespace {

// out[t] over a 3-D tensor (x fastest): a pass along axis ax maps extent ni -> no with the 1-D
// matrix M (row r: M[r * ld + i]), or its transpose (tr). dims: current extents (e0, e1, e2).
__device__ void axis_pass(const double *in, double *out, const double *Mat, int ld, bool tr, int ax, int e0, int e1,
                          int e2, int no, bool acc) {
  const int o0 = ax == 0 ? no : e0, o1 = ax == 1 ? no : e1, o2 = ax == 2 ? no : e2;
  const int ni = ax == 0 ? e0 : (ax == 1 ? e1 : e2);
  const int total = o0 * o1 * o2;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int i0 = t % o0, i1 = (t / o0) % o1, i2 = t / (o0 * o1);
    const int r = ax == 0 ? i0 : (ax == 1 ? i1 : i2);
    double s = 0.0;
    for (int k = 0; k < ni; ++k) {
      const int j0 = ax == 0 ? k : i0, j1 = ax == 1 ? k : i1, j2 = ax == 2 ? k : i2;
      const double w = tr ? Mat[k * ld + r] : Mat[r * ld + k];
      s += w * in[j0 + e0 * (j1 + e1 * j2)];
    }
    out[t] = acc ? out[t] + s : s;
  }
  __syncthreads();
}

struct NsLayout {
  int coef, ecoef, f, X, Y, Z, uv, r, re, total;
};

__host__ __device__ inline NsLayout ns_layout(int n, int qmax) {
  NsLayout L;
  // every work array holds a volume tensor of up to qmax^3 points or 3 face tensors of qmax^2
  const int n3 = n * n * n, P = qmax * qmax * qmax > 3 * qmax * qmax ? qmax * qmax * qmax : 3 * qmax * qmax;
  int o = 0;
  L.coef = o; o += 3 * n3;
  L.ecoef = o; o += 24;
  L.f = o; o += P;
  L.X = o; o += P;
  L.Y = o; o += P;
  L.Z = o; o += P;
  L.uv = o; o += 3 * P;
  L.r = o; o += 3 * n3;
  L.re = o; o += 24;
  L.total = o;
  return L;
}

template <int MODE>
__global__ void ns_op_kernel(MeshView<double> m, const double *__restrict__ in, double dt_over_cr,
                             double *__restrict__ y, int qmax) {
  extern __shared__ double sm[];
  const Basis<double> &B = *m.basis;
  const int n = m.n1, nn = n * n, n3 = nn * n, c = blockIdx.x, tid = threadIdx.x;
  const NsLayout L = ns_layout(n, qmax);
  double *coef = sm + L.coef, *ec = sm + L.ecoef, *f = sm + L.f, *X = sm + L.X, *Y = sm + L.Y, *Z = sm + L.Z;
  double *r = sm + L.r, *re = sm + L.re, *uv = sm + L.uv;
  const int e = m.enr[c];   // switched-on enrichment of this cell, or -1
  const bool enr = e >= 0;
  const int sl = m.slot ? m.slot[c] : -1;
  constexpr int NIN = MODE == NS_GRAD ? 1 : 3;
  for (int t = tid; t < NIN * n3; t += blockDim.x) coef[t] = in[(size_t)c * NIN * n3 + t];
  for (int t = tid; t < 24; t += blockDim.x) {
    ec[t] = (MODE != NS_GRAD && enr) ? in[3 * m.np + (size_t)e * 3 * m.nef + (m.nef == 8 ? t : t >> 3)] : 0.0;
    re[t] = 0.0;
  }
  for (int t = tid; t < 3 * n3; t += blockDim.x) r[t] = 0.0;
  __syncthreads();
  const int sx = (enr && m.full_q) ? QSET_WALL : QSET_LIN, sy = enr ? QSET_WALL : QSET_LIN;
  const int q0 = B.q[sx], q1 = B.q[sy], P = q0 * q1 * q0;
  const double *S0 = B.S[sx], *D0 = B.D[sx], *Sy = B.S[sy], *Dy = B.D[sy];
  const bool curved = m.geo == GEO_CURVED;
  const int col = curved ? metric_col(m, c) : 0;
  const double h[3] = {m.hx, curved ? 1.0 : m.hy[(c / m.nx) % m.ny], m.hz};
  const double hinv[3] = {1.0 / h[0], 1.0 / h[1], 1.0 / h[2]}, hvol = h[0] * h[1] * h[2];   // once per cell
  auto metric = [&](int t, double Ji[3][3], double &dV) {
    const int i0 = t % q0, i1 = (t / q0) % q1, i2 = t / (q0 * q1);
    const double w3 = B.w[sx][i0] * B.w[sy][i1] * B.w[sx][i2];
    if (curved) {
      double det;
      load_rec(vol_rec(m, B, col, sx, sy, i0, i1), Ji, det);
      dV = fabs(det) * w3;
    } else {
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Ji[a][b] = a == b ? hinv[a] : 0.0;
      dV = hvol * w3;
    }
  };
  const double *wtv = enr ? m.wt_vol[0] + (size_t)e * m.nvol[0] * WT : nullptr;
  auto xi_of = [&](int t, double xi[3]) {
    const int i0 = t % q0, i1 = (t / q0) % q1, i2 = t / (q0 * q1);
    xi[0] = B.x[sx][i0]; xi[1] = B.x[sy][i1]; xi[2] = B.x[sx][i2];
  };

  // ---- values at the points: f(t) ----
  if (MODE == NS_GRAD) {
    axis_pass(coef, X, S0, n, false, 0, n, n, n, q0, false);
    axis_pass(X, Y, Sy, n, false, 1, q0, n, n, q1, false);
    axis_pass(Y, Z, S0, n, false, 2, q0, q1, n, q0, false);
    for (int t = tid; t < P; t += blockDim.x) {
      double Ji[3][3], dV;
      metric(t, Ji, dV);
      f[t] = -dV * Z[t];
    }
    __syncthreads();
  } else {
    // point values of u (NS_TAU) or the curl (NS_CURL) accumulate in uv
    for (int t = tid; t < P; t += blockDim.x) f[t] = 0.0;
    if (MODE == NS_CURL)
      for (int t = tid; t < 3 * P; t += blockDim.x) uv[t] = 0.0;
    for (int a = 0; a < 3; ++a) {
      for (int d = 0; d < (MODE == NS_TAU ? 1 : 3); ++d) {
        if (MODE == NS_CURL && !curved && d == a) continue;     // the curl has no du_a/dx_a
        constexpr bool DER = MODE == NS_CURL;
        axis_pass(coef + a * n3, X, (DER && d == 0) ? D0 : S0, n, false, 0, n, n, n, q0, false);
        axis_pass(X, Y, (DER && d == 1) ? Dy : Sy, n, false, 1, q0, n, n, q1, false);
        axis_pass(Y, Z, (DER && d == 2) ? D0 : S0, n, false, 2, q0, q1, n, q0, false);
        for (int t = tid; t < P; t += blockDim.x) {
          if (MODE == NS_TAU) {
            uv[a * P + t] = Z[t];
          } else if (MODE == NS_CURL) {
            double Ji[3][3], dV;
            metric(t, Ji, dV);
            // du_a/dx_e += J^-1[d][e] du_a/dxi_d, into curl = (du2/dx1 - du1/dx2, du0/dx2 - du2/dx0, ...)
            for (int e2 = 0; e2 < 3; ++e2) {
              const double g = Ji[d][e2] * Z[t];
              if (a == 2 && e2 == 1) uv[t] += g;
              if (a == 1 && e2 == 2) uv[t] -= g;
              if (a == 0 && e2 == 2) uv[P + t] += g;
              if (a == 2 && e2 == 0) uv[P + t] -= g;
              if (a == 1 && e2 == 0) uv[2 * P + t] += g;
              if (a == 0 && e2 == 1) uv[2 * P + t] -= g;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int t = tid; t < P; t += blockDim.x) {
      double Ji[3][3], dV;
      metric(t, Ji, dV);
      double uu[3] = {0.0, 0.0, 0.0}, ge[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      if (MODE == NS_TAU) for (int a = 0; a < 3; ++a) uu[a] = uv[a * P + t];
      if (enr) {
        double xi[3], N[8], dN[8][3];
        xi_of(t, xi);
        q1_weights(xi, N, dN);
        const double *w = wtv + (size_t)t * WT;
        for (int v = 0; v < 8; ++v) {
          double g[3];
          ref_to_phys(Ji, dN[v], g);
          for (int a = 0; a < 3; ++a) {
            uu[a] += w[0] * N[v] * ec[a * 8 + v];
            for (int e2 = 0; e2 < 3; ++e2) ge[a][e2] += ec[a * 8 + v] * (w[0] * g[e2] + N[v] * w[1 + e2]);
          }
        }
      }
      if (MODE == NS_TAU) {
        f[t] = dV * sqrt(uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]);
      } else {
        uv[t] = dV * (uv[t] + ge[2][1] - ge[1][2]);
        uv[P + t] = dV * (uv[P + t] + ge[0][2] - ge[2][0]);
        uv[2 * P + t] = dV * (uv[2 * P + t] + ge[1][0] - ge[0][1]);
      }
    }
    __syncthreads();
  }

  if constexpr (MODE == NS_TAU) {
    // tau_D = (int |u| / vol) vol^(1/3) dt / Cr, sums in a fixed order
    if (tid < 32) {
      double s = 0.0, v = 0.0;
      for (int t = tid; t < P; t += 32) {
        double Ji[3][3], dV;
        metric(t, Ji, dV);
        s += f[t];
        v += dV;
      }
      for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        v += __shfl_down_sync(0xffffffffu, v, o);
      }
      if (tid == 0) y[c] = (s / v) * cbrt(v) * dt_over_cr;
    }
    return;
  }

  if constexpr (MODE == NS_CURL) {
    // values: r_a += sum_t dV curl_a(t) phi(t); enriched: sum_t dV curl_a psi N_v
    for (int a = 0; a < 3; ++a) {
      axis_pass(uv + a * P, Y, S0, n, true, 2, q0, q1, q0, n, false);
      axis_pass(Y, X, Sy, n, true, 1, q0, q1, n, n, false);
      axis_pass(X, r + a * n3, S0, n, true, 0, q0, n, n, n, true);
    }
    if (enr && tid < 24) {
      const int a = tid / 8, v = tid % 8;
      double sacc = 0.0;
      for (int t = 0; t < P; ++t) {
        double xi[3], N[8], dN[8][3];
        xi_of(t, xi);
        q1_weights(xi, N, dN);
        sacc += uv[a * P + t] * wtv[(size_t)t * WT] * N[v];
      }
      re[tid] += sacc;
    }
    __syncthreads();
  }
  if constexpr (MODE != NS_TAU && MODE != NS_CURL) {
  // ---- volume: r_a += sum_t f(t) J^-1[d][a] d phi / d xi_d ----
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) {
      if (!curved && d != a) continue;   // boxes: J^-1 is diagonal
      for (int t = tid; t < P; t += blockDim.x) {
        double Ji[3][3], dV;
        metric(t, Ji, dV);
        Z[t] = f[t] * Ji[d][a];
      }
      __syncthreads();
      axis_pass(Z, Y, d == 2 ? D0 : S0, n, true, 2, q0, q1, q0, n, false);
      axis_pass(Y, X, d == 1 ? Dy : Sy, n, true, 1, q0, q1, n, n, false);
      axis_pass(X, r + a * n3, d == 0 ? D0 : S0, n, true, 0, q0, n, n, n, true);
    }
  // enriched test functions: sum_t f(t) d(psi N_v)/dx_a
  if (enr && tid < 24) {
    const int a = tid / 8, v = tid % 8;
    double s = 0.0;
    for (int t = 0; t < P; ++t) {
      double Ji[3][3], dV, xi[3], N[8], dN[8][3], g[3];
      metric(t, Ji, dV);
      xi_of(t, xi);
      q1_weights(xi, N, dN);
      ref_to_phys(Ji, dN[v], g);
      const double *w = wtv + (size_t)t * WT;
      s += f[t] * (w[0] * g[a] + N[v] * w[1 + a]);
    }
    re[tid] += s;
  }
  __syncthreads();
  }
  if constexpr (MODE != NS_TAU) {

  // ---- faces (gradient only): (v, {{p}} n) ----
  if (MODE == NS_GRAD) {
    for (int fc = 0; fc < 6; ++fc) {
      const int d = fc >> 1, side = fc & 1, nb = neighbour(m, c, fc);
      int t1, t2;
      face_axes(d, t1, t2);
      const bool enr_nb = nb >= 0 ? m.enr[nb] >= 0 : enr;
      const bool enr_any = enr || enr_nb;
      const int s1 = ((t1 == 1 || m.full_q) && enr_any) ? QSET_WALL : QSET_LIN;
      const int s2 = ((t2 == 1 || m.full_q) && enr_any) ? QSET_WALL : QSET_LIN;
      const int p1 = B.q[s1], p2 = B.q[s2], FP = p1 * p2;
      // own and neighbour face layers (node index along d: side ? n-1 : 0, and the opposite)
      double *lo = X, *ln = X + nn, *tmp = Y, *g = Z;   // X holds 2 nn <= P, Y p1 n, Z 3 FP + FP
      for (int t = tid; t < nn; t += blockDim.x) {
        const int i1 = t % n, i2 = t / n;
        int id[3], idn[3];
        id[d] = side ? n - 1 : 0; id[t1] = i1; id[t2] = i2;
        idn[d] = side ? 0 : n - 1; idn[t1] = i1; idn[t2] = i2;
        lo[t] = coef[id[0] + n * (id[1] + n * id[2])];
        ln[t] = nb >= 0 ? in[(size_t)nb * n3 + idn[0] + n * (idn[1] + n * idn[2])] : 0.0;
      }
      __syncthreads();
      // face values of both sides at the face points, then the coefficients g_a = dA {{p}} n_a
      for (int t = tid; t < FP; t += blockDim.x) {
        const int a1 = t % p1, a2 = t / p1;
        double po = 0.0, pn = 0.0;
        for (int i2 = 0; i2 < n; ++i2)
          for (int i1 = 0; i1 < n; ++i1) {
            const double w = B.S[s1][a1 * n + i1] * B.S[s2][a2 * n + i2];
            po += w * lo[i1 + n * i2];
            pn += w * ln[i1 + n * i2];
          }
        const double avg = nb >= 0 ? 0.5 * (po + pn) : po;
        double nrm[3], dA;
        const double ww = B.w[s1][a1] * B.w[s2][a2];
        if (curved) {
          double Ji[3][3], det;
          load_rec(face_rec(m, B, col, d, side, s1, s2, a1, a2), Ji, det);
          const double gl = sqrt(Ji[d][0] * Ji[d][0] + Ji[d][1] * Ji[d][1] + Ji[d][2] * Ji[d][2]);
          for (int k = 0; k < 3; ++k) nrm[k] = (side ? 1.0 : -1.0) * Ji[d][k] / gl;
          dA = fabs(det) * gl * ww;
        } else {
          for (int k = 0; k < 3; ++k) nrm[k] = k == d ? (side ? 1.0 : -1.0) : 0.0;
          dA = h[t1] * h[t2] * ww;
        }
        for (int a = 0; a < 3; ++a) g[a * FP + t] = dA * avg * nrm[a];
      }
      __syncthreads();
      // standard test functions on the face layer: r_a[layer] += S_s1^T S_s2^T g_a
      for (int a = 0; a < 3; ++a) {
        for (int t = tid; t < p2 * n; t += blockDim.x) {   // tmp[a2][i1] = sum_a1 S_s1[a1][i1] g[a1][a2]
          const int i1 = t % n, a2 = t / n;
          double s = 0.0;
          for (int a1 = 0; a1 < p1; ++a1) s += B.S[s1][a1 * n + i1] * g[a * FP + a1 + p1 * a2];
          tmp[t] = s;
        }
        __syncthreads();
        for (int t = tid; t < nn; t += blockDim.x) {
          const int i1 = t % n, i2 = t / n;
          double s = 0.0;
          for (int a2 = 0; a2 < p2; ++a2) s += B.S[s2][a2 * n + i2] * tmp[i1 + n * a2];
          int id[3];
          id[d] = side ? n - 1 : 0; id[t1] = i1; id[t2] = i2;
          r[a * n3 + id[0] + n * (id[1] + n * id[2])] += s;
        }
        __syncthreads();
      }
      // enriched test functions: psi N_v at the face points
      if (enr && tid < 24) {
        const int a = tid / 8, v = tid % 8;
        const double *wf = m.wt_face[0] + ((size_t)e * 6 + fc) * m.fpmax[0] * WT;
        double s = 0.0;
        for (int t = 0; t < FP; ++t) {
          const int a1 = t % p1, a2 = t / p1;
          double xi[3], N[8], dN[8][3];
          xi[d] = side; xi[t1] = B.x[s1][a1]; xi[t2] = B.x[s2][a2];
          q1_weights(xi, N, dN);
          s += g[a * FP + t] * wf[(size_t)t * WT] * N[v];
        }
        re[tid] += s;
      }
      __syncthreads();
    }
  }

  // ---- outputs ----
  for (int t = tid; t < 3 * n3; t += blockDim.x) y[(size_t)c * 3 * n3 + t] = r[t];
  if (enr) {
    if (m.nef == 8) {
      for (int t = tid; t < 24; t += blockDim.x) y[3 * m.np + (size_t)e * 24 + t] = re[t];
    } else if (tid < 3) {
      double s = 0.0;
      for (int v = 0; v < 8; ++v) s += re[tid * 8 + v];
      y[3 * m.np + (size_t)e * 3 + tid] = s;
    }
  } else if (sl >= 0) {
    for (int t = tid; t < 3 * m.nef; t += blockDim.x) y[3 * m.np + (size_t)sl * 3 * m.nef + t] = 0.0;
  }
  }
}

// Value and physical gradient of a velocity-type field at wall-face point (a1, a2) of the face
// xi_1 = side (Gauss-Lobatto nodes: the face trace is the node row jend), enrichment included.
__device__ void wall_face_state(const Basis<double> &B, int sq, const double *su, const double *ce, const double *wt,
                                const double xi[3], const double Ji[3][3], int n, int a1, int a2, int side,
                                double U[3], double G[3][3]) {
  const double *S = B.S[sq], *D = B.D[sq], *de = B.dend[side];
  const int n3 = n * n * n, jend = side ? n - 1 : 0;
  for (int a = 0; a < 3; ++a) {
    const double *ua = su + a * n3;
    double v = 0.0, g[3] = {0.0, 0.0, 0.0};
    for (int l = 0; l < n; ++l)
      for (int ii = 0; ii < n; ++ii) {
        const double ul = ua[ii + n * (jend + n * l)];
        v += S[a1 * n + ii] * S[a2 * n + l] * ul;
        g[0] += D[a1 * n + ii] * S[a2 * n + l] * ul;
        g[2] += S[a1 * n + ii] * D[a2 * n + l] * ul;
        double s1 = 0.0;
        for (int jj = 0; jj < n; ++jj) s1 += de[jj] * ua[ii + n * (jj + n * l)];
        g[1] += S[a1 * n + ii] * S[a2 * n + l] * s1;
      }
    U[a] = v;
    ref_to_phys(Ji, g, G[a]);
  }
  if (wt) {
    double N[8], dN[8][3];
    q1_weights(xi, N, dN);
    for (int v = 0; v < 8; ++v) {
      double gN[3];
      ref_to_phys(Ji, dN[v], gN);
      for (int a = 0; a < 3; ++a) {
        U[a] += ce[a * 8 + v] * wt[0] * N[v];
        for (int d = 0; d < 3; ++d) G[a][d] += ce[a * 8 + v] * (wt[0] * gN[d] + N[v] * wt[1 + d]);
      }
    }
  }
}

// Wall integrals (q, g) of the high-order pressure Neumann data (eq. bc_d_pres), added to y:
// g = -(sum_i beta_i (div(u_i x u_i) + nu curl omega_i) - f) . n at the (k+1)^2 Gauss points of each
// wall face (interior traces), one CTA per wall face (wall, i, k).
__global__ void pressure_neumann_kernel(MeshView<double> m, const double *__restrict__ u0,
                                        const double *__restrict__ w0, double b0, const double *__restrict__ u1,
                                        const double *__restrict__ w1, double b1, double f0, double f1, double f2,
                                        double nu, const double *__restrict__ wt_face, int fpmax,
                                        double *__restrict__ y) {
  const Basis<double> &B = *m.basis;
  const int n = m.n1, nn = n * n, n3 = nn * n;
  const int b = blockIdx.x, wall = b / (m.nx * m.nz), r = b % (m.nx * m.nz), i = r % m.nx, kz = r / m.nx;
  const int j = wall ? m.ny - 1 : 0, c = i + m.nx * (j + m.ny * kz), side = wall, jend = side ? n - 1 : 0;
  __shared__ double su[4][3 * NMAX * NMAX * NMAX], ce[4][24], gp[QMAX * QMAX];
  const double *src[4] = {u0, w0, u1, w1};
  const int e = m.enr[c];
  for (int fld = 0; fld < 4; ++fld) {
    const double *v = src[fld];
    for (int t = threadIdx.x; t < 3 * n3; t += blockDim.x) su[fld][t] = v ? v[(size_t)c * 3 * n3 + t] : 0.0;
    for (int t = threadIdx.x; t < 24; t += blockDim.x)
      ce[fld][t] = (v && e >= 0) ? v[3 * m.np + (size_t)e * 3 * m.nef + (m.nef == 8 ? t : t >> 3)] : 0.0;
  }
  __syncthreads();
  // k+1 points per direction; q_w on the wall faces of enriched cells under the q_w^3 rule
  const int sq = (m.full_q && e >= 0) ? QSET_WALL : QSET_LIN, pq = B.q[sq];
  for (int t = threadIdx.x; t < pq * pq; t += blockDim.x) {
    const int a1 = t % pq, a2 = t / pq;
    const double xi[3] = {B.x[sq][a1], (double)side, B.x[sq][a2]};
    double Ji[3][3], det;
    if (m.geo == GEO_CURVED) {
      load_rec(face_rec(m, B, metric_col(m, c), 1, side, sq, sq, a1, a2), Ji, det);
    } else {
      const double h[3] = {m.hx, m.hy[j], m.hz};
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) Ji[p][q] = p == q ? 1.0 / h[p] : 0.0;
      det = h[0] * h[1] * h[2];
    }
    const double gl = sqrt(Ji[1][0] * Ji[1][0] + Ji[1][1] * Ji[1][1] + Ji[1][2] * Ji[1][2]);
    const double sg = side ? 1.0 : -1.0;
    const double nrm[3] = {sg * Ji[1][0] / gl, sg * Ji[1][1] / gl, sg * Ji[1][2] / gl};
    const double dA = fabs(det) * gl * B.w[sq][a1] * B.w[sq][a2];
    const double *wt = e >= 0 ? wt_face + (((size_t)e * 6 + 2 + side) * fpmax + t) * WT : nullptr;
    double acc[3] = {-f0, -f1, -f2};
    for (int h2 = 0; h2 < 2; ++h2) {
      const double beta = h2 ? b1 : b0;
      if (beta == 0.0 || !src[2 * h2]) continue;
      double U[3], G[3][3], W[3], GW[3][3];
      wall_face_state(B, sq, su[2 * h2], ce[2 * h2], wt, xi, Ji, n, a1, a2, side, U, G);
      wall_face_state(B, sq, su[2 * h2 + 1], ce[2 * h2 + 1], wt, xi, Ji, n, a1, a2, side, W, GW);
      const double dv = G[0][0] + G[1][1] + G[2][2];
      const double cw[3] = {GW[2][1] - GW[1][2], GW[0][2] - GW[2][0], GW[1][0] - GW[0][1]};
      for (int a = 0; a < 3; ++a) {
        const double conv = U[a] * dv + U[0] * G[a][0] + U[1] * G[a][1] + U[2] * G[a][2];
        acc[a] += beta * (conv + nu * cw[a]);
      }
    }
    gp[t] = -dA * (acc[0] * nrm[0] + acc[1] * nrm[1] + acc[2] * nrm[2]);
  }
  __syncthreads();
  const double *S = B.S[sq];
  for (int t = threadIdx.x; t < nn; t += blockDim.x) {
    const int i1 = t % n, i2 = t / n;
    double acc = 0.0;
    for (int a2 = 0; a2 < pq; ++a2)
      for (int a1 = 0; a1 < pq; ++a1) acc += S[a1 * n + i1] * S[a2 * n + i2] * gp[a1 + pq * a2];
    y[(size_t)c * n3 + i1 + n * (jend + n * i2)] += acc;
  }
}

}  // namespace

cudaError_t launch_pressure_neumann(dgw_mesh *M, const double *u0, const double *w0, double b0, const double *u1,
                                    const double *w1, double b1, const double *f, double *y, cudaStream_t s) {
  note_launch();
  pressure_neumann_kernel<<<2 * M->P.nx * M->P.nz, 64, 0, s>>>(M->v64, u0, w0, b0, u1, w1, b1, f[0], f[1], f[2],
                                                               M->P.nu, M->v64.wt_face[0], M->v64.fpmax[0], y);
  return cudaGetLastError();
}

cudaError_t launch_ns_op(int mode, dgw_mesh *M, const double *in, double dt_over_cr, double *y, cudaStream_t s) {
  const int n = M->n1;
  const int qmax = std::max(n, M->basis64.q[QSET_WALL]);
  const NsLayout L = ns_layout(n, qmax);
  const size_t smem = (size_t)L.total * sizeof(double);
  cudaError_t e = cudaSuccess;
  note_launch();
  if (mode == NS_GRAD) {
    e = cudaFuncSetAttribute(ns_op_kernel<NS_GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) ns_op_kernel<NS_GRAD><<<M->nc, 128, smem, s>>>(M->v64, in, dt_over_cr, y, qmax);

  } else if (mode == NS_TAU) {
    e = cudaFuncSetAttribute(ns_op_kernel<NS_TAU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) ns_op_kernel<NS_TAU><<<M->nc, 128, smem, s>>>(M->v64, in, dt_over_cr, y, qmax);
  } else {
    e = cudaFuncSetAttribute(ns_op_kernel<NS_CURL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) ns_op_kernel<NS_CURL><<<M->nc, 128, smem, s>>>(M->v64, in, dt_over_cr, y, qmax);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace dgw
