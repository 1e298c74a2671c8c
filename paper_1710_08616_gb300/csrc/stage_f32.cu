// The float instantiation of the RK3 stage kernel (see stage_impl.cuh).
#include "stage_impl.cuh"

namespace asuca {
template cudaError_t launch_stage<float>(const StageParams<float> &, int, cudaStream_t);
template cudaError_t encode_stage_map<float>(CUtensorMap *, void *, int, int, int, int);
}  // namespace asuca
