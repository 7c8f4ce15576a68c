// Solver workspace and multigrid interface (internal).
#pragma once

#include "dgw_internal.h"

namespace dgw {

// device scalar slots of the CG recurrences
enum { SC_RZ = 0, SC_RZNEW, SC_DQ, SC_RR, SC_BB, SC_TMP, SC_RZOLD, SC_RN, SC_COUNT = 8 };

// blocks of the first stage of the two-stage reductions (reduce_to writes this many partial sums)
constexpr int RED_BLOCKS = 304;   // 2 x 152 SMs

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
  // mixed mode: FP32 inner PCG vectors (r and z alias the finest level's b and x) and the captured
  // FP32 V-cycle with its mean projection
  float *d32 = nullptr, *q32 = nullptr, *e32 = nullptr, *zold32 = nullptr;
  cudaGraphExec_t vgraph32 = nullptr;
  unsigned long long vgraph32_launches = 0, vgraph32_dofs = 0;
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
// FP32 hierarchy (mode 1): the finest level's right-hand side and iterate buffers, and one V-cycle
// b0 -> x0 without scaling
cudaError_t mg_level0_f32(dgw_solver *S, float **b0, float **x0);
cudaError_t mg_vcycle_f32(dgw_solver *S, cudaStream_t s);
void mg_free(dgw_solver *S);
dgw_solver *get_solver(dgw_mesh *M);
int mg_levels(dgw_solver *S);
int mg_describe(dgw_solver *S, double *lmax, int *cells, int max_levels);

}  // namespace dgw
