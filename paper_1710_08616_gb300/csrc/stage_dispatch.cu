// Stage launch by tile height (the grid's tuned choice; 8 for FP64 and for
// branch-recording launches).
#include "common.cuh"

namespace asuca {

template <>
cudaError_t launch_stage<float>(const StageParams<float> &p, int nf, cudaStream_t s) {
    switch (p.ty) {
        case 4: return launch_stage_ty<float, 4>(p, nf, s);
        case 16: return launch_stage_ty<float, 16>(p, nf, s);
        default: return launch_stage_ty<float, 8>(p, nf, s);
    }
}

template <>
cudaError_t launch_stage<double>(const StageParams<double> &p, int nf, cudaStream_t s) {
    return launch_stage_ty<double, 8>(p, nf, s);
}

}  // namespace asuca
