// The double instantiation of the dataflow step kernel (see dataflow.cuh).
#include "dataflow.cuh"

namespace asuca {
template cudaError_t launch_dataflow_ty<double, 8>(const DfParams<double> &, int, int, int, cudaStream_t, int *);
}  // namespace asuca
