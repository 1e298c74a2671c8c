// The float stage kernels with 16-row tiles (see stage_impl.cuh).
#include "stage_impl.cuh"

namespace asuca {
template cudaError_t launch_stage_ty<float, 16>(const StageParams<float> &, int, cudaStream_t);
}  // namespace asuca
