// The double ensemble kernel with 8-row tiles (see ensemble.cuh).
#include "ensemble.cuh"

namespace asuca {
template cudaError_t launch_ensemble_ty<double, 8>(const EnsParams<double> &, int, int, int, cudaStream_t, int *);
}  // namespace asuca
