// The float stage kernels with 8-row tiles (see stage_impl.cuh).
#include "stage_impl.cuh"

namespace asuca {
template cudaError_t launch_stage_ty<float, 8>(const StageParams<float> &, int, cudaStream_t);
template cudaError_t encode_stage_map<float>(CUtensorMap *, void *, int, int, int, int, int);
template cudaError_t encode_user_maps<float>(CUtensorMap *, const void *, const void *, const void *, int, int, int,
                                            int, int);
}  // namespace asuca
