// Jacobi diagonal of the SIPG Laplacian (eq. ipflux) on curved cells: a(phi_i, phi_i) with the
// volume term and the own-side face terms (homogeneous Neumann walls carry none; where a periodic
// direction holds a single cell, the face also couples phi_i with its own trace on the far side).
// One thread per DoF evaluates the 1-D factors of phi_i at every point directly: a setup kernel,
// run once per mesh and multigrid level.
#include "metric.cuh"

namespace dgw {

__global__ void curved_diag_kernel(MeshView<double> m, double *__restrict__ dg) {
  const Basis<double> &B = *m.basis;
  const int n = m.n1, n3 = n * n * n;
  const long gid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (gid >= (long)m.nc * n3) return;
  const int c = (int)(gid / n3), i = (int)(gid % n3);
  const int id[3] = {i % n, (i / n) % n, i / (n * n)};
  const int col = metric_col(m, c);
  const int q = B.q[QSET_LIN];
  const double *S = B.S[QSET_LIN], *D = B.D[QSET_LIN], *w = B.w[QSET_LIN];
  double v = 0.0;
  for (int q2 = 0; q2 < q; ++q2)
    for (int q1 = 0; q1 < q; ++q1)
      for (int q0 = 0; q0 < q; ++q0) {
        double Ji[3][3], det;
        load_rec(vol_rec(m, B, col, QSET_LIN, QSET_LIN, q0, q1), Ji, det);
        const double s0 = S[q0 * n + id[0]], s1 = S[q1 * n + id[1]], s2 = S[q2 * n + id[2]];
        const double gr[3] = {D[q0 * n + id[0]] * s1 * s2, s0 * D[q1 * n + id[1]] * s2, s0 * s1 * D[q2 * n + id[2]]};
        double g[3];
        ref_to_phys(Ji, gr, g);
        v += fabs(det) * w[q0] * w[q1] * w[q2] * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
      }
  for (int f = 0; f < 6; ++f) {
    const int nb = neighbour(m, c, f);
    if (nb < 0) continue;
    const int d = f >> 1, side = f & 1;
    int t1, t2;
    t1 = d == 0 ? 1 : 0;
    t2 = d == 2 ? 1 : 2;
    const double tau = fmax(m.tau[c], m.tau[nb]);
    const double sgn = side ? 1.0 : -1.0;
    // 1-D factors of phi_i along d on the face (own side) and on the far side of the same cell
    const double Ld = id[d] == (side ? n - 1 : 0) ? 1.0 : 0.0, dLd = B.dend[side][id[d]];
    const double Lo = id[d] == (side ? 0 : n - 1) ? 1.0 : 0.0, dLo = B.dend[1 - side][id[d]];
    for (int a2 = 0; a2 < q; ++a2)
      for (int a1 = 0; a1 < q; ++a1) {
        double Ji[3][3], det;
        load_rec(face_rec(m, B, col, d, side, QSET_LIN, QSET_LIN, a1, a2), Ji, det);
        const double nrm = sqrt(Ji[d][0] * Ji[d][0] + Ji[d][1] * Ji[d][1] + Ji[d][2] * Ji[d][2]);
        const double nv[3] = {sgn * Ji[d][0] / nrm, sgn * Ji[d][1] / nrm, sgn * Ji[d][2] / nrm};
        const double dA = fabs(det) * nrm * w[a1] * w[a2];
        const double St1 = S[a1 * n + id[t1]], Dt1 = D[a1 * n + id[t1]];
        const double St2 = S[a2 * n + id[t2]], Dt2 = D[a2 * n + id[t2]];
        double gr[3], g[3];
        gr[d] = dLd * St1 * St2; gr[t1] = Ld * Dt1 * St2; gr[t2] = Ld * St1 * Dt2;
        ref_to_phys(Ji, gr, g);
        const double phi = Ld * St1 * St2;
        const double dn = g[0] * nv[0] + g[1] * nv[1] + g[2] * nv[2];
        double po = 0.0, dno = 0.0;
        if (nb == c) {
          double Jo[3][3], deto;
          load_rec(face_rec(m, B, col, d, 1 - side, QSET_LIN, QSET_LIN, a1, a2), Jo, deto);
          gr[d] = dLo * St1 * St2; gr[t1] = Lo * Dt1 * St2; gr[t2] = Lo * St1 * Dt2;
          ref_to_phys(Jo, gr, g);
          po = Lo * St1 * St2;
          dno = g[0] * nv[0] + g[1] * nv[1] + g[2] * nv[2];
        }
        const double jump = phi - po;
        v -= dA * (0.5 * dn * jump + phi * (0.5 * (dn + dno) - tau * jump));
      }
  }
  dg[gid] = v;
}

cudaError_t launch_curved_diagonal(const MeshView<double> &m, double *dg, cudaStream_t s) {
  const long total = (long)m.nc * m.n1 * m.n1 * m.n1;
  const int threads = 128;
  const long blocks = (total + threads - 1) / threads;
  note_launch();
  curved_diag_kernel<<<(unsigned)blocks, threads, 0, s>>>(m, dg);
  return cudaGetLastError();
}

}  // namespace dgw
