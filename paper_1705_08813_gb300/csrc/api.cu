// C ABI entry points: mesh construction, operator applies, eddy-viscosity update.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "dgw_internal.h"

namespace dgw {

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};
static std::atomic<unsigned long long> g_dofs{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launch_counter() { return g_launches.load(std::memory_order_relaxed); }
void note_dofs(long long n) { g_dofs.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
unsigned long long dof_counter() { return g_dofs.load(std::memory_order_relaxed); }

dgw_status set_error(dgw_status s, const std::string &msg) {
  g_last_error = msg;
  return s;
}

dgw_status cuda_check(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return DGW_OK;
  return set_error(DGW_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename X>
static X *dalloc(dgw_mesh *M, size_t count, cudaError_t *err) {
  void *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&p, count * sizeof(X));
  if (e != cudaSuccess) { *err = e; return nullptr; }
  M->allocs.push_back(p);
  M->hbm_bytes += count * sizeof(X);
  return static_cast<X *>(p);
}

template <typename X>
static X *upload(dgw_mesh *M, const X *h, size_t count, cudaStream_t s, cudaError_t *err) {
  X *d = dalloc<X>(M, count, err);
  if (!d) return nullptr;
  if (count) {
    cudaError_t e = cudaMemcpyAsync(d, h, count * sizeof(X), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { *err = e; return nullptr; }
  }
  return d;
}

static void free_mesh(dgw_mesh *M);

template <typename T>
static void fill_view(dgw_mesh *M, MeshView<T> &v) {
  v.nx = M->P.nx; v.ny = M->P.ny; v.nz = M->P.nz;
  v.n1 = M->n1; v.nc = M->nc; v.ne = M->ne;
  v.np = M->np; v.nu = M->nu; v.nef = M->nef; v.full_q = M->P.full_quadrature ? 1 : 0;
  v.hx = (T)(M->P.lx / M->P.nx);
  v.hz = (T)(M->P.lz / M->P.nz);
  v.visc = (T)M->P.nu;
  // box-kernel rows: no enrichment slot in the row (layers are whole rows); the rows next to the
  // layers are included when their y-faces take the standard point sets (no q_w^3 rule): the box
  // kernels add the neighbour's enrichment on those faces
  const int nx = M->P.nx, ny = M->P.ny;
  int nb = 0, nt = 0;
  while (nb < ny && M->enr[(size_t)nx * nb] >= 0) ++nb;
  while (nt < ny - nb && M->enr[(size_t)nx * (ny - 1 - nt)] >= 0) ++nt;
  const int pad = M->P.full_quadrature ? 1 : 0;
  int lo = nb == 0 ? 0 : nb + pad, hi = nt == 0 ? ny : ny - nt - pad;
  if (M->P.geometry != 0 || lo >= hi) lo = hi = ny;
  v.plain_lo = lo;
  v.plain_hi = hi;
  int slo = nb, shi = ny - nt;
  if (M->P.geometry != 0 || slo >= shi) slo = shi = ny;
  v.std_lo = slo;
  v.std_hi = shi;
}

}  // namespace dgw

using namespace dgw;

void dgw_helm_free(dgw_mesh *M);

extern "C" {

const char *dgw_last_error(void) { return g_last_error.c_str(); }

void dgw_counters(unsigned long long *kernel_launches, unsigned long long *dof_applies) {
  if (kernel_launches) *kernel_launches = g_launches.load(std::memory_order_relaxed);
  if (dof_applies) *dof_applies = g_dofs.load(std::memory_order_relaxed);
}

dgw_status dgw_mesh_create(const dgw_mesh_params *P, void *stream, dgw_mesh_t *out) {
  if (!P || !out) return set_error(DGW_EINVAL, "dgw_mesh_create: null argument");
  *out = nullptr;
  if (P->degree < 1 || P->degree > 5) return set_error(DGW_EINVAL, "dgw_mesh_create: degree must be in 1..5");
  if (P->nx < 1 || P->ny < 1 || P->nz < 1) return set_error(DGW_EINVAL, "dgw_mesh_create: cell counts must be >= 1");
  if (P->geometry != 0 && P->geometry != 1)
    return set_error(DGW_EINVAL, "dgw_mesh_create: geometry must be 0 (channel) or 1 (bump)");
  if (P->n_layers < 0 || 2 * P->n_layers > P->ny)
    return set_error(DGW_EINVAL, "dgw_mesh_create: need 0 <= n_layers and 2*n_layers <= ny");
  if (P->enrich_l != 0 && P->enrich_l != 1) return set_error(DGW_EINVAL, "dgw_mesh_create: enrich_l must be 0 or 1");
  if (P->full_quadrature != 0 && P->full_quadrature != 1)
    return set_error(DGW_EINVAL, "dgw_mesh_create: full_quadrature must be 0 or 1");
  if (P->q_wall < 1 || P->q_wall > QW_MAX) return set_error(DGW_EINVAL, "dgw_mesh_create: q_wall must be in 1..10");
  if (!(P->lx > 0 && P->ly > 0 && P->lz > 0 && P->stretch_gamma > 0 && P->nu > 0 && P->tau_w > 0))
    return set_error(DGW_EINVAL, "dgw_mesh_create: lengths, gamma, nu and tau_w must be positive");
  if (P->wall_law != 0 && P->wall_law != 1) return set_error(DGW_EINVAL, "dgw_mesh_create: wall_law must be 0 or 1");
  long long ncl = (long long)P->nx * P->ny * P->nz;
  if (ncl > (1LL << 26)) return set_error(DGW_EINVAL, "dgw_mesh_create: too many cells");
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0)
    return set_error(DGW_ECUDA, "dgw_mesh_create: no CUDA device");
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaError_t ce = box_constants_init(); ce != cudaSuccess) return cuda_check(ce, "dgw_mesh_create");
  if (cudaError_t ce = curved_constants_init(); ce != cudaSuccess) return cuda_check(ce, "dgw_mesh_create");
  dgw_mesh *M = new dgw_mesh();
  M->P = *P;
  const int k = P->degree, n = k + 1;
  M->n1 = n;
  M->nc = (int)ncl;
  M->np = (long)M->nc * n * n * n;
  const int nx = P->nx, ny = P->ny, nz = P->nz;
  const bool curved = P->geometry == 1;
  const int qc = (3 * k) / 2 + 1;
  fill_basis<double>(k, qc, P->q_wall, &M->basis64);
  fill_basis<float>(k, qc, P->q_wall, &M->basis32);
  // vertex rows of the tanh-graded channel (Sec. 5.1)
  M->yv.resize(ny + 1);
  for (int j = 0; j <= ny; ++j)
    M->yv[j] = 0.5 * P->ly * std::tanh(P->stretch_gamma * (2.0 * j / ny - 1.0)) / std::tanh(P->stretch_gamma);
  M->hy.resize(ny);
  for (int j = 0; j < ny; ++j) M->hy[j] = M->yv[j + 1] - M->yv[j];
  // penalty tau_IP = (k+1)^2 A/V per cell, interior faces weighted 1/2, wall faces 1
  BoxGeometry geo;
  CurvedHost cg;
  if (curved) {
    curved_geometry(*P, nx, ny, nz, k, M->basis64, cg);
    M->tau.resize(M->nc);
    for (int c = 0; c < M->nc; ++c) M->tau[c] = cg.tau[c % (nx * ny)];
    M->cxn = cg.xn;
    M->cyn = cg.yn;
  } else {
    box_geometry(k, nx, ny, nz, P->lx, P->lz, M->yv, geo);
    M->tau = geo.tau;
  }
  // enriched cells: bottom rows then top rows, lexicographic (x fastest, then z)
  M->enr.assign(M->nc, -1);
  const int L = P->n_layers;
  int ne = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (int j = 0; j < ny; ++j) {
      const bool rowb = j < L, rowt = j >= ny - L;
      if (!(pass == 0 ? rowb : (rowt && !rowb))) continue;
      for (int kz = 0; kz < nz; ++kz)
        for (int i = 0; i < nx; ++i) M->enr[i + nx * (j + ny * kz)] = ne++;
    }
  M->ne = ne;
  M->nef = P->enrich_l == 0 ? 1 : 8;
  M->nu = 3 * M->np + 3L * M->nef * ne;
  M->enr_cell.resize(std::max(ne, 1));
  for (int c = 0; c < M->nc; ++c)
    if (M->enr[c] >= 0) M->enr_cell[M->enr[c]] = c;
  M->ywall.resize(8 * std::max(ne, 1));
  M->tauv.resize(8 * std::max(ne, 1));
  M->tsrc.resize(8 * std::max(ne, 1));
  M->dye.resize(std::max(ne, 1));
  // each vertex also records the wall node (index wall * nx * nz + i + nx * k) that defines its
  // distance; a nodal wall shear stress reaches the vertex from that node
  for (int e = 0; e < ne; ++e) {
    const int c = M->enr_cell[e], i = c % nx, j = (c / nx) % ny, kz = c / (nx * ny);
    if (!curved) {
      for (int v = 0; v < 8; ++v) {
        const double y = M->yv[j + ((v >> 1) & 1)];
        const double db = y - M->yv[0], dt = M->yv[ny] - y;
        M->ywall[8 * e + v] = std::min(db, dt);   // closest wall node
        M->tauv[8 * e + v] = P->tau_w;
        M->tsrc[8 * e + v] = (db <= dt ? 0 : nx * nz) + (i + (v & 1)) % nx + nx * ((kz + (v >> 2)) % nz);
      }
      M->dye[e] = M->hy[j];
      continue;
    }
    // curved: distance to the closest vertex of either wall (the map does not depend on z, so the
    // closest wall vertex lies in the vertex's own z plane), and the mean of the four edges
    // crossing the cell in the wall-normal direction
    for (int v = 0; v < 8; ++v) {
      double xv, yv;
      bump_point(*P, nx, ny, i + (v & 1), j + ((v >> 1) & 1), &xv, &yv);
      double best = 1e300;
      int src = 0;
      for (int wi = 0; wi <= nx; ++wi)
        for (int wj = 0; wj <= ny; wj += ny) {
          double xw, yw;
          bump_point(*P, nx, ny, wi, wj, &xw, &yw);
          const double d2 = (xw - xv) * (xw - xv) + (yw - yv) * (yw - yv);
          if (d2 < best) {
            best = d2;
            src = (wj ? nx * nz : 0) + wi % nx + nx * ((kz + (v >> 2)) % nz);
          }
        }
      M->ywall[8 * e + v] = std::sqrt(best);
      M->tauv[8 * e + v] = P->tau_w;
      M->tsrc[8 * e + v] = src;
    }
    double len = 0.0;
    for (int o = 0; o < 2; ++o) {
      double x0, y0, x1, y1;
      bump_point(*P, nx, ny, i + o, j, &x0, &y0);
      bump_point(*P, nx, ny, i + o, j + 1, &x1, &y1);
      len += std::sqrt((x1 - x0) * (x1 - x0) + (y1 - y0) * (y1 - y0));
    }
    M->dye[e] = 0.5 * len;
  }
  M->has32 = (P->precision_mask & 2) != 0;
  cudaError_t err = cudaSuccess;
  fill_view(M, M->v64);
  fill_view(M, M->v32);
  for (int sidx = 0; sidx < NQSET; ++sidx) { M->v64.q[sidx] = M->basis64.q[sidx]; M->v32.q[sidx] = M->basis32.q[sidx]; }
  std::vector<float> hy32(M->hy.begin(), M->hy.end()), tau32(M->tau.begin(), M->tau.end());
  M->hy_dev64 = upload(M, M->hy.data(), ny, s, &err);
  M->v64.hy = M->hy_dev64;
  M->v64.tau = upload(M, M->tau.data(), M->nc, s, &err);
  M->v64.enr = upload(M, M->enr.data(), M->nc, s, &err);
  M->v32.enr = M->v64.enr;
  M->slot_dev = upload(M, M->enr.data(), M->nc, s, &err);
  M->v64.slot = M->v32.slot = M->slot_dev;
  M->v64.basis = upload(M, &M->basis64, 1, s, &err);
  M->v64.geo = M->v32.geo = curved ? GEO_CURVED : GEO_BOX;
  if (curved) {
    auto up2 = [&](const std::vector<double> &h, const double **d64, const float **d32) {
      *d64 = upload(M, h.data(), h.size(), s, &err);
      if (M->has32) {
        std::vector<float> f(h.begin(), h.end());
        *d32 = upload(M, f.data(), f.size(), s, &err);
      }
    };
    for (int t = 0; t < NMVOL; ++t)
      if (!cg.mvol[t].empty()) up2(cg.mvol[t], &M->v64.mvol[t], &M->v32.mvol[t]);
    for (int t = 0; t < NQSET; ++t) up2(cg.mxf[t], &M->v64.mxf[t], &M->v32.mxf[t]);
    for (int t = 0; t < NQSET; ++t)
      if (!cg.myf[t].empty()) up2(cg.myf[t], &M->v64.myf[t], &M->v32.myf[t]);
    up2(cg.lvol, &M->v64.lvol, &M->v32.lvol);
    up2(cg.lface, &M->v64.lface, &M->v32.lface);
  } else {
    std::vector<double> rops;
    box_rowscal(geo, rops);
    std::vector<float> rops32(rops.begin(), rops.end());
    M->v64.rowops = upload(M, rops.data(), rops.size(), s, &err);
    M->v32.rowops = upload(M, rops32.data(), rops32.size(), s, &err);
  }
  if (M->has32) {
    M->v32.hy = upload(M, hy32.data(), ny, s, &err);
    M->v32.tau = upload(M, tau32.data(), M->nc, s, &err);
    M->v32.basis = upload(M, &M->basis32, 1, s, &err);
  }
  M->enr_cell_dev = upload(M, M->enr_cell.data(), M->enr_cell.size(), s, &err);
  M->wall_ywall_dev = upload(M, M->ywall.data(), M->ywall.size(), s, &err);
  M->wall_tauv_dev = upload(M, M->tauv.data(), M->tauv.size(), s, &err);
  M->tsrc_dev = upload(M, M->tsrc.data(), M->tsrc.size(), s, &err);
  {
    // wall-nearest enriched cell of every enriched cell's column (the switch-off decides per column)
    std::vector<int> ws(std::max(ne, 1), 0);
    const int L = P->n_layers;
    for (int e = 0; e < ne; ++e) {
      const int c = M->enr_cell[e], i = c % nx, j = (c / nx) % ny, kz = c / (nx * ny);
      ws[e] = M->enr[i + nx * ((j < L ? 0 : ny - 1) + ny * kz)];
    }
    M->wslot_dev = upload(M, ws.data(), ws.size(), s, &err);
  }
  M->wall_mom_dev = dalloc<double>(M, (size_t)2 * nx * nz * 16, &err);
  M->dye_dev = upload(M, M->dye.data(), M->dye.size(), s, &err);
  const int qw = P->q_wall;
  for (int cls = 0; cls < 2; ++cls) {
    const int qi = cls == 0 ? n : qc;
    const int nvol = P->full_quadrature ? qw * qw * qw : qi * qi * qw;
    const int fpmax = P->full_quadrature ? qw * qw : std::max(qw * qi, qi * qi);
    M->v64.nvol[cls] = M->v32.nvol[cls] = nvol;
    M->v64.fpmax[cls] = M->v32.fpmax[cls] = fpmax;
    M->v64.wt_vol[cls] = dalloc<double>(M, (size_t)ne * nvol * WT, &err);
    M->v64.wt_face[cls] = dalloc<double>(M, (size_t)ne * 6 * fpmax * WT, &err);
    if (M->has32) {
      M->v32.wt_vol[cls] = dalloc<float>(M, (size_t)ne * nvol * WT, &err);
      M->v32.wt_face[cls] = dalloc<float>(M, (size_t)ne * 6 * fpmax * WT, &err);
    }
  }
  const size_t nv0 = (size_t)ne * M->v64.nvol[0], nf0 = (size_t)ne * 6 * M->v64.fpmax[0];
  M->aux_vol = dalloc<double>(M, nv0 * 3, &err);    // (y_h, y+, l_mix^2) per point
  M->aux_face = dalloc<double>(M, nf0 * 3, &err);
  M->v64.nut_vol = dalloc<double>(M, nv0, &err);
  M->v64.nut_face = dalloc<double>(M, nf0, &err);
  if (M->has32) {
    M->v32.nut_vol = dalloc<float>(M, nv0, &err);
    M->v32.nut_face = dalloc<float>(M, nf0, &err);
  }
  if (err != cudaSuccess) {
    free_mesh(M);
    return set_error(err == cudaErrorMemoryAllocation ? DGW_ENOMEM : DGW_ECUDA,
                     std::string("dgw_mesh_create: ") + cudaGetErrorString(err));
  }
  // nu_t = 0 until the first update
  cudaMemsetAsync((void *)M->v64.nut_vol, 0, nv0 * sizeof(double), s);
  cudaMemsetAsync((void *)M->v64.nut_face, 0, nf0 * sizeof(double), s);
  if (M->has32) {
    cudaMemsetAsync((void *)M->v32.nut_vol, 0, nv0 * sizeof(float), s);
    cudaMemsetAsync((void *)M->v32.nut_face, 0, nf0 * sizeof(float), s);
  }
  err = launch_wall_tables(M, s);
  if (err == cudaSuccess && M->has32)
    for (int cls = 0; cls < 2 && err == cudaSuccess; ++cls) {
      err = launch_to_float(M->v64.wt_vol[cls], const_cast<float *>(M->v32.wt_vol[cls]),
                            (size_t)ne * M->v64.nvol[cls] * WT, s);
      if (err == cudaSuccess)
        err = launch_to_float(M->v64.wt_face[cls], const_cast<float *>(M->v32.wt_face[cls]),
                              (size_t)ne * 6 * M->v64.fpmax[cls] * WT, s);
    }
  // Jacobi diagonal
  if (curved) {
    if (err == cudaSuccess) M->diag64 = dalloc<double>(M, M->np, &err);
    if (err == cudaSuccess) M->diag32 = dalloc<float>(M, M->np, &err);
    if (err == cudaSuccess) err = launch_curved_diagonal(M->v64, M->diag64, s);
    if (err == cudaSuccess) err = launch_to_float(M->diag64, M->diag32, M->np, s);
  } else {
    std::vector<double> dg;
    laplace_diagonal(geo, M->basis64, dg);
    std::vector<float> dg32(dg.begin(), dg.end());
    if (err == cudaSuccess) M->diag64 = upload(M, dg.data(), dg.size(), s, &err);
    if (err == cudaSuccess) M->diag32 = upload(M, dg32.data(), dg32.size(), s, &err);
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) {
    free_mesh(M);
    return set_error(err == cudaErrorMemoryAllocation ? DGW_ENOMEM : DGW_ECUDA,
                     std::string("dgw_mesh_create: ") + cudaGetErrorString(err));
  }
  *out = M;
  return DGW_OK;
}

dgw_status dgw_mesh_info(dgw_mesh_t M, long *n_p, long *n_u, long *n_enriched, size_t *hbm_bytes) {
  if (!M) return set_error(DGW_EINVAL, "dgw_mesh_info: null mesh");
  if (n_p) *n_p = M->np;
  if (n_u) *n_u = M->nu;
  if (n_enriched) *n_enriched = M->ne;
  if (hbm_bytes) *hbm_bytes = M->hbm_bytes;
  return DGW_OK;
}

dgw_status dgw_mesh_node_coords(dgw_mesh_t M, double *xyz) {
  if (!M || !xyz) return set_error(DGW_EINVAL, "dgw_mesh_node_coords: null argument");
  double z[NMAX], w[NMAX];
  lobatto_nodes(M->n1, z);
  (void)w;
  const int n = M->n1, nx = M->P.nx, ny = M->P.ny, nz = M->P.nz;
  const double hx = M->P.lx / nx, hz = M->P.lz / nz;
  const bool curved = M->P.geometry == 1;
  for (int kz = 0; kz < nz; ++kz)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t c = i + (size_t)nx * (j + (size_t)ny * kz);
        const size_t col = (size_t)(i + nx * j) * n * n;
        for (int c3 = 0; c3 < n; ++c3)
          for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
              double *X = xyz + 3 * (c * n * n * n + a + n * (b + n * c3));
              X[0] = curved ? M->cxn[col + a + n * b] : hx * (i + z[a]);
              X[1] = curved ? M->cyn[col + a + n * b] : M->yv[j] + M->hy[j] * z[b];
              X[2] = hz * (kz + z[c3]);
            }
      }
  return DGW_OK;
}

dgw_status dgw_update_eddy_viscosity(dgw_mesh_t M, const double *u, void *stream) {
  if (!M || !u) return set_error(DGW_EINVAL, "dgw_update_eddy_viscosity: null argument");
  return cuda_check(launch_eddy_viscosity(M, u, (cudaStream_t)stream), "dgw_update_eddy_viscosity");
}


dgw_status dgw_wall_shear_stress(dgw_mesh_t M, const double *u, double *tau_nodes, void *stream) {
  if (!M || !u || !tau_nodes) return set_error(DGW_EINVAL, "dgw_wall_shear_stress: null argument");
  return cuda_check(launch_wall_shear(M, u, tau_nodes, (cudaStream_t)stream), "dgw_wall_shear_stress");
}

// reads the nodal values back and checks that each is finite and > 0 (synchronises s)
static dgw_status check_tau_nodes(dgw_mesh_t M, const double *tau_nodes, cudaStream_t s, const char *name) {
  std::vector<double> h((size_t)2 * M->P.nx * M->P.nz);
  cudaError_t e = cudaMemcpyAsync(h.data(), tau_nodes, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(e, name);
  for (double v : h)
    if (!(v > 0.0) || !std::isfinite(v))
      return set_error(DGW_EINVAL, std::string(name) + ": every nodal value must be finite and > 0");
  return DGW_OK;
}

dgw_status dgw_set_wall_shear_stress(dgw_mesh_t M, const double *tau_nodes, void *stream) {
  if (!M || !tau_nodes) return set_error(DGW_EINVAL, "dgw_set_wall_shear_stress: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  dgw_status st = check_tau_nodes(M, tau_nodes, s, "dgw_set_wall_shear_stress");
  if (st != DGW_OK) return st;
  dgw_helm_free(M);   // the enriched mass blocks of the Helmholtz preconditioner change with tau_w
  return cuda_check(launch_set_tau_nodes(M, tau_nodes, s), "dgw_set_wall_shear_stress");
}

dgw_status dgw_set_enrichment_switch(dgw_mesh_t M, double yplus_off, void *stream) {
  if (!M) return set_error(DGW_EINVAL, "dgw_set_enrichment_switch: null mesh");
  if (!(yplus_off >= 0.0) || !std::isfinite(yplus_off))
    return set_error(DGW_EINVAL, "dgw_set_enrichment_switch: yplus_off must be finite and >= 0");
  M->yp_off = yplus_off;
  dgw_helm_free(M);
  return cuda_check(launch_switch(M, (cudaStream_t)stream), "dgw_set_enrichment_switch");
}

dgw_status dgw_enrichment_active(dgw_mesh_t M, int *active_host, int *n_active, void *stream) {
  if (!M) return set_error(DGW_EINVAL, "dgw_enrichment_active: null mesh");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> enr(M->nc);
  cudaError_t e = cudaMemcpyAsync(enr.data(), M->v64.enr, M->nc * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(e, "dgw_enrichment_active");
  int cnt = 0;
  for (int i = 0; i < M->ne; ++i) {
    const int on = enr[M->enr_cell[i]] >= 0;
    cnt += on;
    if (active_host) active_host[i] = on;
  }
  if (n_active) *n_active = cnt;
  return DGW_OK;
}

dgw_status dgw_project_velocity(dgw_mesh_t M, const double *tau_nodes, const double *u_old, double *u_new,
                                void *stream) {
  if (!M || !tau_nodes || !u_old || !u_new) return set_error(DGW_EINVAL, "dgw_project_velocity: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  // the wall-normal factor of a wall cell's space has k+1 polynomials and 2 (l = 1) or 1 (l = 0)
  // enriched functions; with fewer wall-normal points the discrete cell mass matrix is singular
  if (M->ne > 0 && M->P.q_wall < M->n1 + (M->nef == 8 ? 2 : 1))
    return set_error(DGW_EINVAL, "dgw_project_velocity: q_wall must be at least k+3 (l = 1) or k+2 (l = 0) for "
                                 "the cell mass matrices to be regular");
  dgw_status st = check_tau_nodes(M, tau_nodes, s, "dgw_project_velocity");
  if (st != DGW_OK) return st;
  dgw_helm_free(M);
  int bad = -1;
  st = cuda_check(launch_projection(M, tau_nodes, 1, &u_old, &u_new, s, &bad), "dgw_project_velocity");
  if (st == DGW_OK && bad >= 0)
    return set_error(DGW_EDEVICE, "dgw_project_velocity: the mass matrix of cell " + std::to_string(bad) +
                                      " is not numerically positive definite in the new space");
  return st;
}

dgw_status dgw_apply_gradient(dgw_mesh_t M, const double *p, double *y, void *stream) {
  if (!M || !p || !y) return set_error(DGW_EINVAL, "dgw_apply_gradient: null argument");
  return cuda_check(launch_ns_op(NS_GRAD, M, p, 0.0, y, (cudaStream_t)stream), "dgw_apply_gradient");
}

dgw_status dgw_tau_divdiv(dgw_mesh_t M, const double *u, double dt, double cr, double *tau_d, void *stream) {
  if (!M || !u || !tau_d) return set_error(DGW_EINVAL, "dgw_tau_divdiv: null argument");
  if (!(dt > 0.0) || !(cr > 0.0)) return set_error(DGW_EINVAL, "dgw_tau_divdiv: dt and cr must be positive");
  return cuda_check(launch_ns_op(NS_TAU, M, u, dt / cr, tau_d, (cudaStream_t)stream), "dgw_tau_divdiv");
}

dgw_status dgw_cfl_rate(dgw_mesh_t M, const double *u, double *rate, void *stream) {
  if (!M || !u || !rate) return set_error(DGW_EINVAL, "dgw_cfl_rate: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!M->rate_dev) M->rate_dev = dalloc<double>(M, 1, &e);
  if (e != cudaSuccess) return cuda_check(e, "dgw_cfl_rate");
  e = cudaMemsetAsync(M->rate_dev, 0, sizeof(double), s);
  if (e == cudaSuccess) e = launch_cfl_rate(M->v64, u, M->rate_dev, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rate, M->rate_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_check(e, "dgw_cfl_rate");
}

dgw_status dgw_apply_divdiv(dgw_mesh_t M, const double *tau_d, const double *u, double *y, void *stream) {
  if (!M || !tau_d || !u || !y) return set_error(DGW_EINVAL, "dgw_apply_divdiv: null argument");
  MeshView<double> v = M->v64;
  v.tau_d = tau_d;
  return cuda_check(launch_vector_op<double>(OP_DIVDIV, v, u, y, (cudaStream_t)stream), "dgw_apply_divdiv");
}

dgw_status dgw_apply_curl(dgw_mesh_t M, const double *u, double *y, void *stream) {
  if (!M || !u || !y) return set_error(DGW_EINVAL, "dgw_apply_curl: null argument");
  return cuda_check(launch_ns_op(NS_CURL, M, u, 0.0, y, (cudaStream_t)stream), "dgw_apply_curl");
}

dgw_status dgw_add_pressure_neumann(dgw_mesh_t M, const double *u0, const double *w0, double beta0, const double *u1,
                                    const double *w1, double beta1, const double *force, double *b, void *stream) {
  if (!M || !u0 || !w0 || !force || !b) return set_error(DGW_EINVAL, "dgw_add_pressure_neumann: null argument");
  if (beta1 != 0.0 && (!u1 || !w1)) return set_error(DGW_EINVAL, "dgw_add_pressure_neumann: beta1 needs u1 and w1");
  return cuda_check(launch_pressure_neumann(M, u0, w0, beta0, beta1 != 0.0 ? u1 : nullptr, beta1 != 0.0 ? w1 : nullptr,
                                            beta1, force, b, (cudaStream_t)stream),
                    "dgw_add_pressure_neumann");
}

dgw_status dgw_apply_inverse_mass(dgw_mesh_t M, const double *r, double *x, void *stream) {
  if (!M || !r || !x) return set_error(DGW_EINVAL, "dgw_apply_inverse_mass: null argument");
  if (r == x) return set_error(DGW_EINVAL, "dgw_apply_inverse_mass: r and x must not overlap");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_collocation_inverse_mass(M, r, x, s);
  if (e == cudaSuccess) e = launch_inverse_mass_cells(M, r, x, s);
  if (e == cudaErrorInvalidValue)
    return set_error(DGW_EDEVICE, "dgw_apply_inverse_mass: a wall-cell mass matrix is not numerically positive definite");
  return cuda_check(e, "dgw_apply_inverse_mass");
}

dgw_status dgw_apply_laplace(dgw_mesh_t M, int prec, const void *p, void *y, void *stream) {
  if (!M || !p || !y) return set_error(DGW_EINVAL, "dgw_apply_laplace: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == DGW_FP64)
    return cuda_check(launch_laplace<double>(M->v64, (const double *)p, (double *)y, s), "dgw_apply_laplace");
  if (prec == DGW_FP32) {
    if (!M->has32) return set_error(DGW_EINVAL, "dgw_apply_laplace: mesh built without FP32 tables");
    return cuda_check(launch_laplace<float>(M->v32, (const float *)p, (float *)y, s), "dgw_apply_laplace");
  }
  if (prec == DGW_DF64) {
    if (M->P.geometry != 0) return set_error(DGW_EINVAL, "dgw_apply_laplace: DGW_DF64 needs box cells (geometry 0)");
    return cuda_check(launch_laplace_df(M->v64, (const double *)p, (double *)y, s), "dgw_apply_laplace");
  }
  return set_error(DGW_EINVAL, "dgw_apply_laplace: prec must be DGW_FP64, DGW_FP32 or DGW_DF64");
}

static dgw_status apply_vec(dgw_mesh_t M, int op, int prec, const void *u, void *y, void *stream, const char *name) {
  if (!M || !u || !y) return set_error(DGW_EINVAL, std::string(name) + ": null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == DGW_FP64) return cuda_check(launch_vector_op<double>(op, M->v64, (const double *)u, (double *)y, s), name);
  if (prec == DGW_FP32 && op != OP_DIV) {
    if (!M->has32) return set_error(DGW_EINVAL, std::string(name) + ": mesh built without FP32 tables");
    return cuda_check(launch_vector_op<float>(op, M->v32, (const float *)u, (float *)y, s), name);
  }
  if (prec == DGW_DF64) {
    if (M->P.geometry != 0 || (op != OP_DIV && op != OP_VISC && op != OP_CONV))
      return set_error(DGW_EINVAL, std::string(name) + ": DGW_DF64 needs box cells (geometry 0)");
    return cuda_check(launch_vector_op_df(op, M->v64, (const double *)u, (double *)y, s), name);
  }
  return set_error(DGW_EINVAL, std::string(name) + ": unsupported prec");
}

dgw_status dgw_apply_divergence(dgw_mesh_t M, const double *u, double *b, void *stream) {
  return apply_vec(M, OP_DIV, DGW_FP64, u, b, stream, "dgw_apply_divergence");
}

dgw_status dgw_apply_divergence_prec(dgw_mesh_t M, int prec, const double *u, double *b, void *stream) {
  if (prec != DGW_FP64 && prec != DGW_DF64)
    return set_error(DGW_EINVAL, "dgw_apply_divergence_prec: prec must be DGW_FP64 or DGW_DF64");
  return apply_vec(M, OP_DIV, prec, u, b, stream, "dgw_apply_divergence_prec");
}

dgw_status dgw_apply_convective(dgw_mesh_t M, int prec, const void *u, void *y, void *stream) {
  return apply_vec(M, OP_CONV, prec, u, y, stream, "dgw_apply_convective");
}

dgw_status dgw_apply_viscous(dgw_mesh_t M, int prec, const void *u, void *y, void *stream) {
  return apply_vec(M, OP_VISC, prec, u, y, stream, "dgw_apply_viscous");
}

}  // extern "C"

void dgw_solver_free(dgw_mesh *M);
void dgw_batch_free(dgw_mesh *M);

namespace dgw {
static void free_mesh(dgw_mesh *M) {
  if (!M) return;
  dgw_batch_free(M);
  dgw_solver_free(M);
  dgw_helm_free(M);
  for (void *p : M->allocs) cudaFree(p);
  delete M;
}
}  // namespace dgw

extern "C" dgw_status dgw_mesh_destroy(dgw_mesh_t M) {
  if (!M) return set_error(DGW_EINVAL, "dgw_mesh_destroy: null mesh");
  dgw::free_mesh(M);
  return DGW_OK;
}
