// Geometric multigrid V-cycle used as the lower-level preconditioner M.
#include "device.cuh"

namespace to {

int mg_build(to_problem* P) { return fail(TO_ERR_ARG, "multigrid preconditioner not available in this build"); }
int mg_refresh(to_problem* P, cudaStream_t s) { return fail(TO_ERR_ARG, "multigrid preconditioner not available"); }
int mg_vcycle(to_problem* P, const void* r, void* z, cudaStream_t s) {
    return fail(TO_ERR_ARG, "multigrid preconditioner not available");
}

}  // namespace to
