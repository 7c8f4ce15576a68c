// Cell adjacency of the structured channel and the metric records of curved cells (shared by the
// operator kernels and the curved Jacobi diagonal).
#pragma once

#include "dgw_internal.h"

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

// Metric column of cell c: the curved map is an extrusion along z, so cells (i, j, *) share one
// set of metric records.
template <typename T>
__device__ __forceinline__ int metric_col(const MeshView<T> &m, int c) { return c % (m.nx * m.ny); }

// Volume record at the 2-D point (a0 of the x-set sx, a1 of the y-set sy) of column col.
template <typename T>
__device__ __forceinline__ const T *vol_rec(const MeshView<T> &m, const Basis<T> &B, int col, int sx, int sy, int a0,
                                            int a1) {
  // (wall, wall): the q_w^3 rule, where a wall x-set always comes with a wall y-set
  const int pair = sx == QSET_WALL ? MVOL_WALL_WALL : (sx == QSET_CONV ? 1 : 0) + (sy == QSET_WALL ? 2 : 0);
  const int qx = B.q[sx], qy = B.q[sy];
  return m.mvol[pair] + ((size_t)col * qx * qy + a0 + qx * a1) * MREC;
}

// Record at face point (a1, a2) of the face xi_d = side of column col (t1/t2 sets s1, s2).
template <typename T>
__device__ __forceinline__ const T *face_rec(const MeshView<T> &m, const Basis<T> &B, int col, int d, int side, int s1,
                                             int s2, int a1, int a2) {
  if (d == 0) return m.mxf[s1] + (((size_t)col * 2 + side) * B.q[s1] + a1) * MREC;   // t1 = y
  if (d == 1) return m.myf[s1] + (((size_t)col * 2 + side) * B.q[s1] + a1) * MREC;   // t1 = x
  return vol_rec(m, B, col, s1, s2, a1, a2);                                           // (x, y), z-invariant
}

template <typename T>
__device__ __forceinline__ void load_rec(const T *p, T Ji[3][3], T &det) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) Ji[r][q] = p[r * 3 + q];
  det = p[9];
}

// physical gradient from reference derivatives: g_e = sum_d J^-1[d][e] r_d
template <typename T>
__device__ __forceinline__ void ref_to_phys(const T Ji[3][3], const T r[3], T g[3]) {
#pragma unroll
  for (int e = 0; e < 3; ++e) g[e] = Ji[0][e] * r[0] + Ji[1][e] * r[1] + Ji[2][e] * r[2];
}
// coefficients of the reference derivatives of a test function from a physical vector f:
// c_d = sum_e J^-1[d][e] f_e
template <typename T>
__device__ __forceinline__ void phys_to_ref(const T Ji[3][3], const T f[3], T cf[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) cf[d] = Ji[d][0] * f[0] + Ji[d][1] * f[1] + Ji[d][2] * f[2];
}

}  // namespace dgw
