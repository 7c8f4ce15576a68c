// Solver workspace and multigrid interface (internal).
#pragma once

#include "dgw_internal.h"

namespace dgw {

// device scalar slots of the CG recurrences
enum { SC_RZ = 0, SC_RZNEW, SC_DQ, SC_RR, SC_BB, SC_TMP, SC_RZOLD, SC_COUNT = 8 };

struct MGLevel;

}  // namespace dgw

struct dgw_solver {
  double *b = nullptr, *r = nullptr, *z = nullptr, *d = nullptr, *q = nullptr, *zold = nullptr;
  double *partial = nullptr, *sc = nullptr, *host_sc = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_in = nullptr, ev_out = nullptr;
  cudaStream_t stream = nullptr;   // internal stream (graph capture needs a non-legacy stream)
  // captured V-cycle (fixed buffers r -> z) and the launches / DoF applications one replay adds
  cudaGraphExec_t vgraph = nullptr;
  unsigned long long vgraph_launches = 0, vgraph_dofs = 0;
  // multigrid hierarchy (built on first use per mode)
  bool mg_ready = false;
  int mg_mode = -1;
  int mg_cheb = 0;
  std::vector<dgw::MGLevel *> levels;
};

void dgw_solver_free(dgw_mesh *M);

namespace dgw {

cudaError_t reduce_to(const double *a, const double *b, long n, double *partial, double *sc, int slot, cudaStream_t s);
cudaError_t project_mean(const double *a, double *x, long n, double *partial, double *sc, int slot, cudaStream_t s);
cudaError_t mg_setup(dgw_mesh *M, dgw_solver *S, int mode, int cheb_degree, cudaStream_t s);
cudaError_t mg_vcycle(dgw_mesh *M, dgw_solver *S, int mode, const double *r, double *z, cudaStream_t s);
void mg_free(dgw_solver *S);
dgw_solver *get_solver(dgw_mesh *M);
int mg_levels(dgw_solver *S);
int mg_describe(dgw_solver *S, double *lmax, int *cells, int max_levels);

}  // namespace dgw
