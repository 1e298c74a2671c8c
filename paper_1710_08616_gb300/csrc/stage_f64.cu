// The double instantiation of the RK3 stage kernel (see stage_impl.cuh).
#include "stage_impl.cuh"

namespace asuca {
template cudaError_t launch_stage<double>(const StageParams<double> &, int, cudaStream_t);
template cudaError_t encode_stage_map<double>(CUtensorMap *, void *, int, int, int, int);
}  // namespace asuca
