// Column-pass kernel (grid-stride over columns, one thread per column; the
// per-column code is in column_impl.cuh), the budget reduction, and the
// numerics test hook.
#include "column_impl.cuh"

namespace asuca {

template <typename T, int NF>
__global__ void __launch_bounds__(COL_TPB, 3) column_kernel(const __grid_constant__ ColumnParams<T> p) {
    const long long ncol = p.plane;
    const long long nslots = p.nslots;
    const long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x;

    double bsum[NF + 1];
#pragma unroll
    for (int q = 0; q <= NF; q++) bsum[q] = 0.0;

    for (long long col = slot; col < ncol; col += nslots) {
        ColSum<T> cs[NF];
        column_one<T, NF>(p, col, p.scratch + slot, nslots, cs);
        if (p.budgets) {
#pragma unroll
            for (int f = 0; f < NF; f++) bsum[f] += cs[f].value();
            if (p.precip_col) bsum[NF] += p.precip_col[col];
        }
    }

    if (!p.budgets) return;
    // deterministic block reduction of the per-thread partial sums
    __shared__ double red[COL_TPB];
#pragma unroll
    for (int q = 0; q <= NF; q++) {
        red[threadIdx.x] = bsum[q];
        __syncthreads();
        for (int s = COL_TPB / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) p.partials[(long long)blockIdx.x * (NF + 1) + q] = red[0];
        __syncthreads();
    }
}

// The bottom-up half of the column pass after ColDownHook: back substitution
// from the fused scratch (fscratch_level / fscratch_col), (rho phi)_k = sigma_k z_k
// for rho*theta and every tracer (column_one's bottom-up pass, operation for
// operation), and the column budget partials.  Grid-stride over columns,
// one thread per column.
template <typename T, int NF>
__global__ void __launch_bounds__(COL_TPB, 3) column_up_kernel(const __grid_constant__ ColumnParams<T> p) {
    const long long ncol = p.plane;
    double bsum[NF + 1];
#pragma unroll
    for (int q = 0; q <= NF; q++) bsum[q] = 0.0;

    for (long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x; col < ncol;
         col += (long long)gridDim.x * blockDim.x) {
        ColSum<T> cs[NF];
        column_up_one<T, NF>(p, col, cs);
        if (p.budgets) {
#pragma unroll
            for (int f = 0; f < NF; f++) bsum[f] += cs[f].value();
            if (p.precip_col) bsum[NF] += p.precip_col[col];
        }
    }

    if (!p.budgets) return;
    __shared__ double red[COL_TPB];
#pragma unroll
    for (int q = 0; q <= NF; q++) {
        red[threadIdx.x] = bsum[q];
        __syncthreads();
        for (int s = COL_TPB / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) p.partials[(long long)blockIdx.x * (NF + 1) + q] = red[0];
        __syncthreads();
    }
}

// Sum the block partials in a fixed order, scale the field sums by dx*dy,
// and flag a non-finite result in the status word.
__global__ void budget_reduce_kernel(const double *partials, int nblocks, int nq, int nf,
                                     double dxdy, double *out, int *status) {
    __shared__ double red[256];
    for (int q = 0; q < nq; q++) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[(long long)b * nq + q];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double v = q < nf ? red[0] * dxdy : red[0];
            out[q] = v;
            if (!isfinite(v) && status) atomicCAS(status, 0, (int)ASUCA_ERR_NONFINITE);
        }
        __syncthreads();
    }
}

// Test hook: the integer-pipe conversions and the double reciprocal on n values.
__global__ void numerics_kernel(const float *in_f, const double *in_d, int n, double *widen,
                                float *narrow, double *rcp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (widen) widen[i] = f2d_bits(in_f[i]);
    if (narrow) narrow[i] = d2f_bits(in_d[i]);
    if (rcp) rcp[i] = rcp_f64(in_d[i]);
}

cudaError_t launch_numerics(const float *in_f, const double *in_d, int n, double *widen, float *narrow,
                            double *rcp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    numerics_kernel<<<(n + 255) / 256, 256, 0, s>>>(in_f, in_d, n, widen, narrow, rcp);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_column(const ColumnParams<T> &p, int nf, int grid, int block, cudaStream_t s) {
    if (block != COL_TPB) return cudaErrorInvalidValue;
    switch (nf) {
#define ASUCA_COL_CASE(N) \
        case N: column_kernel<T, N><<<grid, COL_TPB, 0, s>>>(p); break;
        ASUCA_COL_CASE(2) ASUCA_COL_CASE(3) ASUCA_COL_CASE(4) ASUCA_COL_CASE(5)
        ASUCA_COL_CASE(6) ASUCA_COL_CASE(7) ASUCA_COL_CASE(8) ASUCA_COL_CASE(9)
        ASUCA_COL_CASE(10)
#undef ASUCA_COL_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_column_up(const ColumnParams<T> &p, int nf, int grid, cudaStream_t s) {
    switch (nf) {
#define ASUCA_COLUP_CASE(N) \
        case N: column_up_kernel<T, N><<<grid, COL_TPB, 0, s>>>(p); break;
        ASUCA_COLUP_CASE(2) ASUCA_COLUP_CASE(3) ASUCA_COLUP_CASE(4) ASUCA_COLUP_CASE(5)
        ASUCA_COLUP_CASE(6) ASUCA_COLUP_CASE(7) ASUCA_COLUP_CASE(8) ASUCA_COLUP_CASE(9)
        ASUCA_COLUP_CASE(10)
#undef ASUCA_COLUP_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template cudaError_t launch_column_up<float>(const ColumnParams<float> &, int, int, cudaStream_t);
template cudaError_t launch_column_up<double>(const ColumnParams<double> &, int, int, cudaStream_t);
template cudaError_t launch_column<float>(const ColumnParams<float> &, int, int, int, cudaStream_t);
template cudaError_t launch_column<double>(const ColumnParams<double> &, int, int, int, cudaStream_t);

cudaError_t launch_budget_reduce(const double *partials, int nblocks, int nq, int nf, double dxdy,
                                 double *out, int *status, cudaStream_t s) {
    budget_reduce_kernel<<<1, 256, 0, s>>>(partials, nblocks, nq, nf, dxdy, out, status);
    return cudaGetLastError();
}

}  // namespace asuca
