// The float ensemble kernel with 4-row tiles (see ensemble.cuh).
#include "ensemble.cuh"

namespace asuca {
template cudaError_t launch_ensemble_ty<float, 4>(const EnsParams<float> &, int, int, int, cudaStream_t, int *);

}  // namespace asuca
