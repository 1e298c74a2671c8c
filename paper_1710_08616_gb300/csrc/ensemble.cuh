// Ensemble of members with uneven horizontal domains advanced in one
// persistent, cooperative launch.  For each step the kernel runs three stage
// phases, the second and third carrying the top-down half of the column pass
// (FactorHook, SweepHook), and one back-substitution phase; a phase walks a
// flattened list of work items
// (member, tile) or (member, column), dealt round-robin to the resident CTAs,
// and ends at a device-wide barrier.  Members never share a tile, so each
// member's result equals its own single-member step bit for bit.
//
// The barrier is a generation counter in the workspace.  Its wait is bounded
// (about one second of wall time); a CTA that gives up writes
// ASUCA_ERR_TIMEOUT to the status word and leaves the kernel, and so do the
// others when their own waits run out.
#pragma once

#include "ensemble_params.cuh"
#include "smem_attr.cuh"
#include "fused_impl.cuh"

namespace asuca {

__device__ __forceinline__ bool ens_barrier(unsigned *count, unsigned *gen, unsigned target, int *status) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        volatile unsigned *vgen = gen;
        const unsigned g0 = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u) + 1u;
        int ok = 1;
        if (arrived == target) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (*vgen == g0) {
                if (global_ns() - t0 > 1000000000ull) {
                    ok = 0;
                    if (status) atomicCAS(status, 0, (int)ASUCA_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(200);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <typename T>
__device__ __forceinline__ int member_of(const EnsMember<T> *m, int nm, long long idx, bool by_tile) {
    int lo = 0, hi = nm - 1;
    while (lo < hi) {   // last member whose first index <= idx
        const int mid = (lo + hi + 1) >> 1;
        const long long first = by_tile ? m[mid].tile0 : m[mid].col0;
        if (first <= idx) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Shared memory of the ensemble kernel: the stage tile's, copies of the
// current tile's stage parameters and of the scalar head of its column
// parameters (everything before the per-level arrays), which the tile reads
// many times per level, then the per-level records of the column pass (nz of
// them, the largest level count of the members).
template <typename T, int NF, int TYV>
struct EnsSmem {
    static constexpr size_t SP = FusedSmem<T, NF, TYV>::TILE;
    static constexpr size_t CP = SP + (sizeof(StageParams<T>) + 127) / 128 * 128;
    static constexpr size_t HEAD = (offsetof(ColumnParams<T>, dzT) + 7) / 8 * 8;
    static constexpr size_t TAB = (CP + HEAD + 127) / 128 * 128;
    static size_t bytes(int nz) { return TAB + (size_t)nz * sizeof(ColLevel<T>); }
    static constexpr size_t MAX_BYTES = TAB + (size_t)MAXNZ * sizeof(ColLevel<T>);
};

// 8-byte copy of bytes (a multiple of 8) by the CTA's threads
__device__ __forceinline__ void cta_copy8(void *dst, const void *src, size_t bytes, int tid, int nthr) {
    long long *d = reinterpret_cast<long long *>(dst);
    const long long *q = reinterpret_cast<const long long *>(src);
    for (size_t i = tid; i < bytes / 8; i += nthr) d[i] = q[i];
}

// The last phase for a column of a member without vertical diffusion (k0 = 0).
// Its factorisation has no coupling (alpha = gamma = 0), so the sweep left
// each field's value after relaxation and sedimentation exactly (widened to
// double) in the scratch; they go to the state as they are.  asuca_step's
// separate column pass skips the solve for such a grid and leaves the same
// values, where the back substitution's scaling by rho dz m (about 1) would
// round them.
template <typename T, int NF>
__device__ __forceinline__ void ens_copy_swept(const ColumnParams<T> &p, long long col) {
    constexpr int NT = NF - 1;
    constexpr int NQ = NF + 1;
    const size_t pl = (size_t)p.plane;
    const size_t ls = (size_t)fscratch_level(p.plane, NQ);
    double *sc = p.scratch + fscratch_col(col, NQ);
    for (int k = 0; k < p.nz; k++) {
        const double *a = fscratch_at(p, sc, k, ls, NQ - 1);
        size_t o = (size_t)k * pl + (size_t)col;
        ASUCA_BC(o, (long long)p.nz * (long long)pl, p.status);
#pragma unroll
        for (int f = 0; f < NT; f++) p.y[f + 1][o] = (T)a[32 * (2 + f)];
    }
}

// Per step: stage 1 (upward march); stage 2 marching downward with the FP64
// factorisation of every column (FactorHook); stage 3 marching downward with
// the relaxation, sedimentation and elimination sweep (SweepHook); then the
// bottom-up back substitution over the flattened columns (ens_copy_swept for a
// member without vertical diffusion).  A tile of stages 2 and 3 first loads
// its member's per-level records into shared memory.
template <typename T, int NF, int LIM, int TYV>
__global__ void __launch_bounds__(32 * TYV, StageShape<T, NF, TYV>::MIN_BLOCKS)
    ensemble_kernel(const __grid_constant__ EnsParams<T> e) {
    using S = StageShape<T, NF, TYV>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    using M = EnsSmem<T, NF, TYV>;
    ColLevel<T> *tab = reinterpret_cast<ColLevel<T> *>(smem_raw + M::TAB);
    StageParams<T> &sp = *reinterpret_cast<StageParams<T> *>(smem_raw + M::SP);
    ColumnParams<T> &cp = *reinterpret_cast<ColumnParams<T> *>(smem_raw + M::CP);   // scalar head only
    static_assert(M::SP % 64 == 0 && sizeof(StageParams<T>) % 8 == 0, "parameter copies");
    const unsigned target = gridDim.x + (unsigned)e.bar_extra;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthr = blockDim.x * blockDim.y;
    const long long nth = (long long)gridDim.x * nthr;
    const long long gtid = (long long)blockIdx.x * nthr + tid;
    for (int n = 0; n < e.nsteps; n++) {
        for (int stg = 0; stg < 3; stg++) {
            bool bad = false;
            for (long long t = blockIdx.x; t < e.total_tiles; t += gridDim.x) {
                const int m = member_of(e.members, e.nmembers, t, true);
                const EnsMember<T> &mb = e.members[m];
                const long long lt = t - mb.tile0;
                const int i0 = (int)(lt % mb.tiles_x) * S::TX, j0 = (int)(lt / mb.tiles_x) * S::TY;
                // the tile's parameters into shared memory (the tensor map is
                // read from the member's copy in global memory)
                __syncthreads();   // the previous tile is done with the copies and the records
                cta_copy8(&sp, &mb.stage[stg], sizeof(StageParams<T>), tid, nthr);
                if (stg > 0) {
                    cta_copy8(&cp, &mb.col, M::HEAD, tid, nthr);
                    fill_col_levels(mb.col, tab, tid, nthr);
                }
                __syncthreads();
                const CUtensorMap *tmap = &mb.stage[stg].tmap;
                if (stg == 0) {
                    bad = stage_tile<T, NF, LIM, false, TYV>(sp, tmap, i0, j0, smem_raw, mb.stage[0].umap);
                } else {
                    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
                    const unsigned own = (i < sp.nx && j < sp.ny) ? (unsigned)(j * sp.nx + i) : 0u;
                    if (stg == 1) {
                        FactorHook<T, NF> h(cp, tab, own);
                        bad = stage_tile_h<T, NF, LIM, false, TYV, true, FactorHook<T, NF>, LAYOUT_PAIR>(
                            sp, tmap, i0, j0, smem_raw, h);
                    } else {
                        SweepHook<T, NF> h(cp, tab, sp.yout[0], own);
                        bad = stage_tile_h<T, NF, LIM, false, TYV, true, SweepHook<T, NF>, LAYOUT_PAIR>(
                            sp, tmap, i0, j0, smem_raw, h);
                    }
                }
                if (bad) break;
            }
            if (bad || !ens_barrier(e.bar_count, e.bar_gen, target, e.status)) return;
        }
        for (long long c = gtid; c < e.total_cols; c += nth) {
            const int m = member_of(e.members, e.nmembers, c, false);
            const EnsMember<T> &mb = e.members[m];
            if (mb.col.do_diff) {
                ColSum<T> cs[NF];
                column_up_one<T, NF>(mb.col, c - mb.col0, cs);
            } else {
                ens_copy_swept<T, NF>(mb.col, c - mb.col0);
            }
        }
        if (!ens_barrier(e.bar_count, e.bar_gen, target, e.status)) return;
    }
}

template <typename T, int NF, int LIM, int TYV>
static cudaError_t ens_launch_lim(const EnsParams<T> &e, int grid, cudaStream_t s, int *grid_out) {
    using S = StageShape<T, NF, TYV>;
    static std::atomic<unsigned long long> attr_done{0};   // devices whose attribute is set
    // tile, parameter copies, per-level records (the attribute allows the largest level count)
    const size_t bytes = EnsSmem<T, NF, TYV>::bytes(e.nzmax);
    const cudaError_t r =
        set_smem_once(ensemble_kernel<T, NF, LIM, TYV>, (int)EnsSmem<T, NF, TYV>::MAX_BYTES, attr_done);
    if (r != cudaSuccess) return r;
    if (grid_out) {   // size query: resident CTAs per SM times SMs
        int per_sm = 0, dev = 0, nsm = 0;
        cudaError_t r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ensemble_kernel<T, NF, LIM, TYV>,
                                                                      32 * S::TY, bytes);
        if (r != cudaSuccess) return r;
        if ((r = cudaGetDevice(&dev)) != cudaSuccess) return r;
        if ((r = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return r;
        *grid_out = per_sm * nsm;
        return cudaSuccess;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32, S::TY);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ensemble_kernel<T, NF, LIM, TYV>, e);
}

template <typename T, int NF, int TYV>
static cudaError_t ens_launch_nf(const EnsParams<T> &e, int lim, int grid, cudaStream_t s, int *grid_out) {
    switch (lim) {
        case ASUCA_LIM_KOREN: return ens_launch_lim<T, NF, ASUCA_LIM_KOREN, TYV>(e, grid, s, grid_out);
        case ASUCA_LIM_LINEAR: return ens_launch_lim<T, NF, ASUCA_LIM_LINEAR, TYV>(e, grid, s, grid_out);
        case ASUCA_LIM_UPWIND1: return ens_launch_lim<T, NF, ASUCA_LIM_UPWIND1, TYV>(e, grid, s, grid_out);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int TYV>
cudaError_t launch_ensemble_ty(const EnsParams<T> &e, int nf, int lim, int grid, cudaStream_t s, int *grid_out) {
    switch (nf) {
        case 2: return ens_launch_nf<T, 2, TYV>(e, lim, grid, s, grid_out);
        case 3: return ens_launch_nf<T, 3, TYV>(e, lim, grid, s, grid_out);
        case 4: return ens_launch_nf<T, 4, TYV>(e, lim, grid, s, grid_out);
        case 5: return ens_launch_nf<T, 5, TYV>(e, lim, grid, s, grid_out);
        case 6: return ens_launch_nf<T, 6, TYV>(e, lim, grid, s, grid_out);
        case 7: return ens_launch_nf<T, 7, TYV>(e, lim, grid, s, grid_out);
        case 8: return ens_launch_nf<T, 8, TYV>(e, lim, grid, s, grid_out);
        case 9: return ens_launch_nf<T, 9, TYV>(e, lim, grid, s, grid_out);
        case 10: return ens_launch_nf<T, 10, TYV>(e, lim, grid, s, grid_out);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace asuca
