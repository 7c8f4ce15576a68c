// Solver workspace and multigrid interface (internal).
#pragma once

#include <chrono>

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
  float *d32 = nullptr, *q32 = nullptr, *e32 = nullptr;
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
// FP32 hierarchy over a block of cols right-hand sides (boxes, dense coarsest solve; otherwise
// cudaErrorNotSupported), its level-0 rhs / iterate blocks (cols x np) and one V-cycle over the
// first ncols columns
cudaError_t mg_batch_create(dgw_mesh *M, int cols, int cheb, cudaStream_t s, void **out);
void mg_batch_free(void *h);
void mg_batch_level0(void *h, float **b0, float **x0);
cudaError_t mg_batch_vcycle(void *h, int ncols, cudaStream_t s);

// ---- block mixed-precision solves (batch.cu): columns of right-hand sides on one mesh
constexpr int kBatchMax = 8;   // columns of a batch
struct BatchColumn {
  const double *b_in = nullptr;    // caller's right-hand side (n_p doubles)
  double *p_out = nullptr;         // caller's solution buffer
  void *caller_stream = nullptr;
  long tag = 0;                    // the caller's identifier of the column
  double rtol = 1e-10;             // the column's target ||b - A p|| / ||b||
  int max_iter = 1000;             // limit on its inner iterations
  bool used = false, finished = false;
  double bnorm = 0.0, rel_residual = 0.0;
  int iterations = 0;              // inner FP32 iterations, all refinement rounds
  dgw_status status = DGW_OK;
  std::chrono::steady_clock::time_point t_admit;
};
struct Batch;
cudaError_t batch_create(dgw_mesh *M, int cap, int cheb, Batch **out);
void batch_destroy(Batch *B);
int batch_active(const Batch *B);   // active columns (they occupy slots 0..active-1)
// a new column in the first free slot (between rounds; the caller checks batch_active < cap)
cudaError_t batch_admit(Batch *B, const BatchColumn &c, cudaStream_t caller);
// one refinement round; finished columns are written to their p_out and appended to done
cudaError_t batch_round(Batch *B, std::vector<BatchColumn> &done);
dgw_solver *get_solver(dgw_mesh *M);
int mg_levels(dgw_solver *S);
int mg_describe(dgw_solver *S, double *lmax, int *cells, int max_levels);

}  // namespace dgw
