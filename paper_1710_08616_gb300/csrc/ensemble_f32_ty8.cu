// The float ensemble kernel with 8-row tiles (see ensemble.cuh).
#include "ensemble.cuh"

namespace asuca {
template cudaError_t launch_ensemble_ty<float, 8>(const EnsParams<float> &, int, int, int, cudaStream_t, int *);

}  // namespace asuca
