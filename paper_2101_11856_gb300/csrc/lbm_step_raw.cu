// Fused step kernels with the RAW collision model (see lbm_step_kernels.cuh).
#include "lbm_step_kernels.cuh"

namespace lbm {
template cudaError_t launch_step_coll<COLL_RAW, false>(int storage, const StepParams &P, bool band, int part, cudaStream_t st);
}  // namespace lbm
