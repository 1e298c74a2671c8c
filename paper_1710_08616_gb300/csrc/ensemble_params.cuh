// Parameters of the ensemble kernel (ensemble.cuh) and its launcher.
#pragma once

#include "common.cuh"

namespace asuca {

// One member, resident in device memory.
template <typename T>
struct EnsMember {
    StageParams<T> stage[3];   // the three stage launches of one step
    ColumnParams<T> col;       // the column pass (scratch and slot count come from EnsParams)
    long long tile0;           // first flattened tile of this member
    long long col0;            // first flattened column of this member
    int tiles_x;
};

template <typename T>
struct EnsParams {
    const EnsMember<T> *members;
    int nmembers, nsteps;
    long long total_tiles, total_cols;
    unsigned *bar_count, *bar_gen;
    int bar_extra;             // 0; a test sets 1 so that the barrier can never complete
    int *status;
    double *scratch;           // column-solve scratch, one slot per thread of the grid
};

// grid_out != nullptr: only store the co-resident grid size in *grid_out
template <typename T>
cudaError_t launch_ensemble(const EnsParams<T> &e, int nf, int lim, int grid, cudaStream_t s, int *grid_out);

}  // namespace asuca
