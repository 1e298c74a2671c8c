// The float instantiation of the ensemble kernel (see ensemble.cuh).
#include "ensemble.cuh"

namespace asuca {
template cudaError_t launch_ensemble<float>(const EnsParams<float> &, int, int, int, cudaStream_t, int *);
}  // namespace asuca
