// Stage 3 with the relaxation, sedimentation and elimination sweep of the
// column pass (the factorisation done in stage 2), float fields, 8-row tiles.
#include "fused_impl.cuh"

namespace asuca {
template <>
cudaError_t launch_stage3_sweep<float>(const FusedParams<float> &p, int nf, cudaStream_t s) {
    return launch_fused_ty<float, 8, 1>(p, nf, s);
}
}  // namespace asuca
