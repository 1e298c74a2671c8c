// The third RK stage fused with the top-down half of the column pass: the
// stage marches its levels from the top down (stage_tile_h with DOWN), and each
// thread hands its column's stage result, level by level, to ColDownHook
// (relaxation, sedimentation, FP64 elimination).  The FP64 elimination thereby
// runs in the same kernel as the FP32 stencil, on the otherwise idle FP64
// pipe; column_up_kernel finishes the column bottom-up.
#pragma once

#include "column_impl.cuh"
#include "smem_attr.cuh"
#include "stage_impl.cuh"

namespace asuca {

template <typename T, int NF, int LIM, int TYV>
__global__ void __launch_bounds__(32 * TYV, StageShape<T, NF, TYV>::MIN_BLOCKS)
    stage3_column_kernel(const __grid_constant__ FusedParams<T> fp) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const StageParams<T> &p = fp.s;
    const int i0 = blockIdx.x * StageShape<T, NF, TYV>::TX, j0 = blockIdx.y * TYV;
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    const unsigned own = (i < p.nx && j < p.ny) ? (unsigned)(j * p.nx + i) : 0u;
    ColDownHook<T, NF> hook(fp.c, p.yout[0], own);
    (void)stage_tile_h<T, NF, LIM, false, TYV, true, ColDownHook<T, NF>, LAYOUT_PAIR>(p, &p.tmap, i0, j0, smem_raw,
                                                                                     hook);
}

template <typename T, int NF, int LIM, int TYV>
static cudaError_t fused_launch_lim(const FusedParams<T> &p, cudaStream_t s) {
    using S = StageShape<T, NF, TYV>;
    static std::atomic<unsigned long long> attr_done{0};   // devices whose attribute is set
    const cudaError_t e = set_smem_once(stage3_column_kernel<T, NF, LIM, TYV>, (int)S::SMEM_BYTES, attr_done);
    if (e != cudaSuccess) return e;
    dim3 block(S::TX, S::TY);
    dim3 grid((p.s.nx + S::TX - 1) / S::TX, (p.s.ny + S::TY - 1) / S::TY);
    stage3_column_kernel<T, NF, LIM, TYV><<<grid, block, S::SMEM_BYTES, s>>>(p);
    return cudaGetLastError();
}

template <typename T, int NF, int TYV>
static cudaError_t fused_launch_nf(const FusedParams<T> &p, cudaStream_t s) {
    switch (p.s.lim) {
        case ASUCA_LIM_KOREN: return fused_launch_lim<T, NF, ASUCA_LIM_KOREN, TYV>(p, s);
        case ASUCA_LIM_LINEAR: return fused_launch_lim<T, NF, ASUCA_LIM_LINEAR, TYV>(p, s);
        case ASUCA_LIM_UPWIND1: return fused_launch_lim<T, NF, ASUCA_LIM_UPWIND1, TYV>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int TYV>
cudaError_t launch_stage3_column_ty(const FusedParams<T> &p, int nf, cudaStream_t s) {
    switch (nf) {
        case 2: return fused_launch_nf<T, 2, TYV>(p, s);
        case 3: return fused_launch_nf<T, 3, TYV>(p, s);
        case 4: return fused_launch_nf<T, 4, TYV>(p, s);
        case 5: return fused_launch_nf<T, 5, TYV>(p, s);
        case 6: return fused_launch_nf<T, 6, TYV>(p, s);
        case 7: return fused_launch_nf<T, 7, TYV>(p, s);
        case 8: return fused_launch_nf<T, 8, TYV>(p, s);
        case 9: return fused_launch_nf<T, 9, TYV>(p, s);
        case 10: return fused_launch_nf<T, 10, TYV>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace asuca
