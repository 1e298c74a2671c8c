// Stage 3 fused with the top-down column pass, double fields, 8-row tiles.
#include "fused_impl.cuh"

namespace asuca {
template <>
cudaError_t launch_stage3_column<double>(const FusedParams<double> &p, int nf, cudaStream_t s) {
    return launch_stage3_column_ty<double, 8>(p, nf, s);
}
}  // namespace asuca
