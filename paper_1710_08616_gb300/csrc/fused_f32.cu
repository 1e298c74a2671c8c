// Stage 3 fused with the whole top-down column pass, float fields, 8-row tiles.
#include "fused_impl.cuh"

namespace asuca {
template <>
cudaError_t launch_stage3_column<float>(const FusedParams<float> &p, int nf, cudaStream_t s) {
    return launch_fused_ty<float, 8, 0>(p, nf, s);
}
}  // namespace asuca
