// Parameters of the ensemble kernel (ensemble.cuh) and its launcher.
#pragma once

#include "common.cuh"

namespace asuca {

// One member, resident in device memory.
template <typename T>
struct EnsMember {
    StageParams<T> stage[3];   // the three stage launches of one step
    ColumnParams<T> col;       // the column pass: its fused scratch and alpha array are the member's own
    long long tile0;           // first flattened tile of this member
    long long col0;            // first flattened column of this member
    int tiles_x;
};

template <typename T>
struct EnsParams {
    const EnsMember<T> *members;
    int nmembers, nsteps;
    int nzmax;                 // the largest level count of the members (sizes the per-level records)
    long long total_tiles, total_cols;
    unsigned *bar_count, *bar_gen;
    int bar_extra;             // 0; a test sets 1 so that the barrier can never complete
    int *status;
};

// grid_out != nullptr: only store the co-resident grid size in *grid_out
template <typename T, int TYV>
cudaError_t launch_ensemble_ty(const EnsParams<T> &e, int nf, int lim, int grid, cudaStream_t s, int *grid_out);

// tile rows ty: 4 or 8 for float, 8 for double
template <typename T>
inline cudaError_t launch_ensemble(const EnsParams<T> &e, int nf, int lim, int ty, int grid, cudaStream_t s,
                                   int *grid_out) {
    if constexpr (sizeof(T) == 4) {
        if (ty == 4) return launch_ensemble_ty<T, 4>(e, nf, lim, grid, s, grid_out);
    }
    return launch_ensemble_ty<T, 8>(e, nf, lim, grid, s, grid_out);
}

}  // namespace asuca
