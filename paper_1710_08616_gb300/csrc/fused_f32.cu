// Stage 3 fused with the top-down column pass, float fields, 8-row tiles.
#include "fused_impl.cuh"

namespace asuca {
template <>
cudaError_t launch_stage3_column<float>(const FusedParams<float> &p, int nf, cudaStream_t s) {
    return launch_stage3_column_ty<float, 8>(p, nf, s);
}
}  // namespace asuca
