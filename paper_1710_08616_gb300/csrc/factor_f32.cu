// Stage 2 with the FP64 factorisation of the column pass, float fields, 8-row tiles.
#include "fused_impl.cuh"

namespace asuca {
template <>
cudaError_t launch_stage2_factor<float>(const FusedParams<float> &p, int nf, cudaStream_t s) {
    return launch_fused_ty<float, 8, 2>(p, nf, s);
}
}  // namespace asuca
