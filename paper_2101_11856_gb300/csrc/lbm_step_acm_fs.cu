// Fused step kernels with the ACM collision model for grids with a free-slip face (see
// lbm_step_kernels.cuh).
#include "lbm_step_kernels.cuh"

namespace lbm {
template cudaError_t launch_step_coll<COLL_ACM, true>(int storage, const StepParams &P, bool band, int part, cudaStream_t st);
}  // namespace lbm
