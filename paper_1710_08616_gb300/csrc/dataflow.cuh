// One domain advanced by a persistent dataflow kernel: every (phase, tile)
// pair of a call -- three RK stages and the column pass per step, on 32 x TY
// tiles of columns -- is a task.  Tasks are handed out by an atomic counter in
// a fixed order in which every task comes after the tasks it reads:
//   a stage task of phase q on tile T reads phase q-1 on T's 3 x 3 tile
//   neighbourhood (the 2-wide halo), a column task reads phase q-1 on T only;
// the order sorts tasks by 2 q + min(r, R - r) for tile row r of R, a
// distance on the periodic ring of rows in which neighbouring rows differ by
// at most one, so tasks of different steps and phases interleave across
// tile rows.  A CTA that takes a task
// waits (bounded, about one second) until its inputs are complete, runs it,
// and publishes the tile's completed-phase count with release semantics.
// The column pass (FP64 elimination, bound by the FP64 pipe) and the stencil
// stages (FP32, bound by issue and memory) thereby run side by side on the
// same SMs instead of one after the other.  Write-after-read hazards on the
// reused stage buffers are covered by the same chain: the writer of a tile's
// buffer depends, through the intermediate phases, on every reader of it.
#pragma once

#include "column_impl.cuh"
#include "smem_attr.cuh"
#include "dataflow_params.cuh"
#include "stage_impl.cuh"

namespace asuca {

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T, int NF, int LIM, int TYV>
__global__ void __launch_bounds__(32 * TYV, StageShape<T, NF, TYV>::MIN_BLOCKS)
    dataflow_kernel(const __grid_constant__ DfParams<T> p) {
    using S = StageShape<T, NF, TYV>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ unsigned task_s;
    __shared__ double red[32 * TYV];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x * blockDim.y;
    const long long gtid = (long long)blockIdx.x * blockDim.x * blockDim.y + tid;
    const unsigned total = (unsigned)p.nslot * (unsigned)p.txn;
    for (;;) {
        if (tid == 0) task_s = atomicAdd(p.counter, 1u);
        __syncthreads();
        const unsigned t = task_s;
        if (t >= total) break;
        const unsigned ent = p.order[t / p.txn];
        const int q = (int)(ent >> 12), r = (int)(ent & 0xfffu), tx = (int)(t % p.txn);
        const int phase = q & 3;
        // ---- wait until the inputs of this task are complete
        int late = 0;
        if (tid < 9) {
            const int dx = tid % 3 - 1, dy = tid / 3 - 1;
            if (phase != 3 || (dx == 0 && dy == 0)) {
                const int nx_ = (tx + dx + p.txn) % p.txn, ny_ = (r + dy + p.tyn) % p.tyn;
                const unsigned *f = p.flags + (size_t)ny_ * p.txn + nx_;
                if (ld_acquire(f) < (unsigned)q) {
                    const uint64_t t0 = global_ns();
                    while (ld_acquire(f) < (unsigned)q) {
                        if (global_ns() - t0 > 1000000000ull) {
                            late = 1;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
            }
        }
        if (__syncthreads_or(late)) {
            if (tid == 0 && p.status) atomicCAS(p.status, 0, (int)ASUCA_ERR_TIMEOUT);
            return;
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");   // inputs read by TMA below
        bool bad = false;
        if (phase < 3) {
            bad = stage_tile<T, NF, LIM, false, TYV>(p.stage[phase], &p.stage[phase].tmap, tx * S::TX, r * TYV,
                                                     smem_raw);
        } else {
            const bool last = q >= p.last_q0;
            const ColumnParams<T> &cp = last ? p.col_last : p.col;
            const int i = tx * S::TX + threadIdx.x, j = r * TYV + threadIdx.y;
            double b[NF + 1];
#pragma unroll
            for (int f = 0; f <= NF; f++) b[f] = 0.0;
            if (i < cp.nx && j < cp.ny) {
                const long long col = (long long)j * cp.nx + i;
                ColSum<T> cs[NF];
                column_one<T, NF>(cp, col, p.scratch + gtid, nth, cs);
                if (cp.budgets) {
#pragma unroll
                    for (int f = 0; f < NF; f++) b[f] = cs[f].value();
                    if (cp.precip_col) b[NF] = cp.precip_col[col];
                }
            }
            if (cp.budgets) {   // fixed-order tree over the tile's columns
                const size_t tile = (size_t)r * p.txn + tx;
#pragma unroll
                for (int f = 0; f <= NF; f++) {
                    red[tid] = b[f];
                    __syncthreads();
                    for (int s = 16 * TYV; s > 0; s >>= 1) {
                        if (tid < s) red[tid] += red[tid + s];
                        __syncthreads();
                    }
                    if (tid == 0) p.partials[tile * (NF + 1) + f] = red[0];
                    __syncthreads();
                }
            }
        }
        if (__syncthreads_or(bad)) return;
        if (tid == 0) {
            __threadfence();
            st_release(p.flags + (size_t)r * p.txn + tx, (unsigned)(q + 1));
        }
    }
}

template <typename T, int NF, int LIM, int TYV>
static cudaError_t df_launch_lim(const DfParams<T> &p, int grid, cudaStream_t s, int *grid_out) {
    using S = StageShape<T, NF, TYV>;
    static std::atomic<unsigned long long> attr_done{0};   // devices whose attribute is set
    const cudaError_t r = set_smem_once(dataflow_kernel<T, NF, LIM, TYV>, (int)S::SMEM_BYTES, attr_done);
    if (r != cudaSuccess) return r;
    if (grid_out) {
        int per_sm = 0, dev = 0, nsm = 0;
        cudaError_t r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dataflow_kernel<T, NF, LIM, TYV>,
                                                                      32 * TYV, S::SMEM_BYTES);
        if (r != cudaSuccess) return r;
        if ((r = cudaGetDevice(&dev)) != cudaSuccess) return r;
        if ((r = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return r;
        *grid_out = per_sm * nsm;
        return cudaSuccess;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32, TYV);
    cfg.dynamicSmemBytes = S::SMEM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // every CTA resident: waits always end
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, dataflow_kernel<T, NF, LIM, TYV>, p);
}

template <typename T, int NF, int TYV>
static cudaError_t df_launch_nf(const DfParams<T> &p, int lim, int grid, cudaStream_t s, int *grid_out) {
    switch (lim) {
        case ASUCA_LIM_KOREN: return df_launch_lim<T, NF, ASUCA_LIM_KOREN, TYV>(p, grid, s, grid_out);
        case ASUCA_LIM_LINEAR: return df_launch_lim<T, NF, ASUCA_LIM_LINEAR, TYV>(p, grid, s, grid_out);
        case ASUCA_LIM_UPWIND1: return df_launch_lim<T, NF, ASUCA_LIM_UPWIND1, TYV>(p, grid, s, grid_out);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int TYV>
cudaError_t launch_dataflow_ty(const DfParams<T> &p, int nf, int lim, int grid, cudaStream_t s, int *grid_out) {
    switch (nf) {
        case 2: return df_launch_nf<T, 2, TYV>(p, lim, grid, s, grid_out);
        case 3: return df_launch_nf<T, 3, TYV>(p, lim, grid, s, grid_out);
        case 4: return df_launch_nf<T, 4, TYV>(p, lim, grid, s, grid_out);
        case 5: return df_launch_nf<T, 5, TYV>(p, lim, grid, s, grid_out);
        case 6: return df_launch_nf<T, 6, TYV>(p, lim, grid, s, grid_out);
        case 7: return df_launch_nf<T, 7, TYV>(p, lim, grid, s, grid_out);
        case 8: return df_launch_nf<T, 8, TYV>(p, lim, grid, s, grid_out);
        case 9: return df_launch_nf<T, 9, TYV>(p, lim, grid, s, grid_out);
        case 10: return df_launch_nf<T, 10, TYV>(p, lim, grid, s, grid_out);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace asuca
