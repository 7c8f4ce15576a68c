// Geometric multigrid preconditioner (built in a later step).
#include "solver.h"

namespace dgw {

cudaError_t mg_setup(dgw_mesh *, dgw_solver *S, int, int, cudaStream_t) {
  S->mg_ready = false;
  return cudaErrorNotSupported;
}
cudaError_t mg_vcycle(dgw_mesh *, dgw_solver *, int, const double *, double *, cudaStream_t) {
  return cudaErrorNotSupported;
}
void mg_free(dgw_solver *S) { S->levels.clear(); S->mg_ready = false; }

}  // namespace dgw
