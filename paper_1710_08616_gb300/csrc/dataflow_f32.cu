// The float instantiation of the dataflow step kernel (see dataflow.cuh).
#include "dataflow.cuh"

namespace asuca {
template cudaError_t launch_dataflow_ty<float, 8>(const DfParams<float> &, int, int, int, cudaStream_t, int *);
}  // namespace asuca
