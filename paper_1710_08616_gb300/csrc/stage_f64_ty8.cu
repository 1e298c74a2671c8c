// The double stage kernels with 8-row tiles (see stage_impl.cuh).
#include "stage_impl.cuh"

namespace asuca {
template cudaError_t launch_stage_ty<double, 8>(const StageParams<double> &, int, cudaStream_t);
template cudaError_t encode_stage_map<double>(CUtensorMap *, void *, int, int, int, int, int);
template cudaError_t encode_user_maps<double>(CUtensorMap *, const void *, const void *, const void *, int, int, int,
                                            int, int);
}  // namespace asuca
