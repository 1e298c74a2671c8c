// The column pass fused into the stage kernels.  The stages march their
// levels from the top down (stage_tile_h with DOWN), and each thread hands its
// column's stage result, level by level, to a hook (column_impl.cuh):
//   * stage3_column_kernel: the third RK stage with ColDownHook (relaxation,
//     sedimentation, FP64 factorisation and elimination), or with SweepHook
//     (relaxation, sedimentation, elimination sweep) when the second stage
//     carried the factorisation;
//   * stage2_factor_kernel: the second RK stage, its result written as usual,
//     with FactorHook (the FP64 factorisation from the density after the step).
// The FP64 work thereby runs in the same kernels as the FP32 stencils, on the
// otherwise idle FP64 pipe; column_up_kernel finishes the column bottom-up.
#pragma once

#include "column_impl.cuh"
#include "smem_attr.cuh"
#include "stage_impl.cuh"

namespace asuca {

// shared memory of a fused stage: the tile's, then the per-level records
template <typename T, int NF, int TYV>
struct FusedSmem {
    static constexpr size_t TILE = (StageShape<T, NF, TYV>::SMEM_BYTES + 127) / 128 * 128;
    static size_t bytes(int nz) { return TILE + (size_t)nz * sizeof(ColLevel<T>); }
    static constexpr size_t MAX_BYTES = TILE + (size_t)MAXNZ * sizeof(ColLevel<T>);
};

template <typename T, int NF, int LIM, int TYV, bool SPLIT>
__global__ void __launch_bounds__(32 * TYV, StageShape<T, NF, TYV>::MIN_BLOCKS)
    stage3_column_kernel(const __grid_constant__ FusedParams<T> fp) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    using S = StageShape<T, NF, TYV>;
    using Hook = typename std::conditional<SPLIT, SweepHook<T, NF>, ColDownHook<T, NF>>::type;
    const StageParams<T> &p = fp.s;
    ColLevel<T> *tab = reinterpret_cast<ColLevel<T> *>(smem_raw + FusedSmem<T, NF, TYV>::TILE);
    fill_col_levels(fp.c, tab, (int)(threadIdx.y * blockDim.x + threadIdx.x), (int)(blockDim.x * blockDim.y));
    __syncthreads();
    const int i0 = blockIdx.x * S::TX, j0 = blockIdx.y * TYV;
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    const unsigned own = (i < p.nx && j < p.ny) ? (unsigned)(j * p.nx + i) : 0u;
    Hook hook(fp.c, tab, p.yout[0], own);
    (void)stage_tile_h<T, NF, LIM, false, TYV, true, Hook, LAYOUT_PAIR>(p, &p.tmap, i0, j0, smem_raw, hook);
}

template <typename T, int NF, int LIM, int TYV>
__global__ void __launch_bounds__(32 * TYV, StageShape<T, NF, TYV>::MIN_BLOCKS)
    stage2_factor_kernel(const __grid_constant__ FusedParams<T> fp) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    using S = StageShape<T, NF, TYV>;
    const StageParams<T> &p = fp.s;
    ColLevel<T> *tab = reinterpret_cast<ColLevel<T> *>(smem_raw + FusedSmem<T, NF, TYV>::TILE);
    fill_col_levels(fp.c, tab, (int)(threadIdx.y * blockDim.x + threadIdx.x), (int)(blockDim.x * blockDim.y));
    __syncthreads();
    const int i0 = blockIdx.x * S::TX, j0 = blockIdx.y * TYV;
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    const unsigned own = (i < p.nx && j < p.ny) ? (unsigned)(j * p.nx + i) : 0u;
    FactorHook<T, NF, true> hook(fp.c, tab, own);
    (void)stage_tile_h<T, NF, LIM, false, TYV, true, FactorHook<T, NF, true>, LAYOUT_PAIR>(p, &p.tmap, i0, j0,
                                                                                         smem_raw, hook);
}

// KIND 0: stage 3 with the whole top-down pass, 1: stage 3 with the sweep
// only, 2: stage 2 with the factorisation
template <typename T, int NF, int LIM, int TYV, int KIND>
static cudaError_t fused_launch_lim(const FusedParams<T> &p, cudaStream_t s) {
    using S = StageShape<T, NF, TYV>;
    using M = FusedSmem<T, NF, TYV>;
    static std::atomic<unsigned long long> attr_done{0};   // devices whose attribute is set
    void (*kern)(const FusedParams<T>);
    if constexpr (KIND == 2) kern = stage2_factor_kernel<T, NF, LIM, TYV>;
    else kern = stage3_column_kernel<T, NF, LIM, TYV, KIND == 1>;
    const cudaError_t e = set_smem_once(kern, (int)M::MAX_BYTES, attr_done);
    if (e != cudaSuccess) return e;
    dim3 block(S::TX, S::TY);
    dim3 grid((p.s.nx + S::TX - 1) / S::TX, (p.s.ny + S::TY - 1) / S::TY);
    kern<<<grid, block, M::bytes(p.s.nz), s>>>(p);
    return cudaGetLastError();
}

template <typename T, int NF, int TYV, int KIND>
static cudaError_t fused_launch_nf(const FusedParams<T> &p, cudaStream_t s) {
    switch (p.s.lim) {
        case ASUCA_LIM_KOREN: return fused_launch_lim<T, NF, ASUCA_LIM_KOREN, TYV, KIND>(p, s);
        case ASUCA_LIM_LINEAR: return fused_launch_lim<T, NF, ASUCA_LIM_LINEAR, TYV, KIND>(p, s);
        case ASUCA_LIM_UPWIND1: return fused_launch_lim<T, NF, ASUCA_LIM_UPWIND1, TYV, KIND>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int TYV, int KIND>
cudaError_t launch_fused_ty(const FusedParams<T> &p, int nf, cudaStream_t s) {
    switch (nf) {
        case 2: return fused_launch_nf<T, 2, TYV, KIND>(p, s);
        case 3: return fused_launch_nf<T, 3, TYV, KIND>(p, s);
        case 4: return fused_launch_nf<T, 4, TYV, KIND>(p, s);
        case 5: return fused_launch_nf<T, 5, TYV, KIND>(p, s);
        case 6: return fused_launch_nf<T, 6, TYV, KIND>(p, s);
        case 7: return fused_launch_nf<T, 7, TYV, KIND>(p, s);
        case 8: return fused_launch_nf<T, 8, TYV, KIND>(p, s);
        case 9: return fused_launch_nf<T, 9, TYV, KIND>(p, s);
        case 10: return fused_launch_nf<T, 10, TYV, KIND>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace asuca
