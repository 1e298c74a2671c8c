// The float stage kernels with 4-row tiles (see stage_impl.cuh).
#include "stage_impl.cuh"

namespace asuca {
template cudaError_t launch_stage_ty<float, 4>(const StageParams<float> &, int, cudaStream_t);
}  // namespace asuca
