// Parameters and launcher of the dataflow step kernel (dataflow.cuh).
#pragma once

#include "common.cuh"

namespace asuca {

template <typename T>
struct DfParams {
    StageParams<T> stage[3];
    ColumnParams<T> col;       // every step but the last
    ColumnParams<T> col_last;  // the last step (budget partials when asked)
    const unsigned *order;     // per wave slot: (phase q << 12) | tile row
    int nslot;                 // Q * R entries of order
    int txn, tyn;              // tiles per row, tile rows
    unsigned *counter;         // task counter
    unsigned *flags;           // per tile: completed phases
    double *scratch;           // column-solve scratch, one slot per thread of the grid
    double *partials;          // per tile: F + 1 budget partials (last step)
    int last_q0;               // first phase of the last step
    int *status;
};


template <typename T, int TYV>
cudaError_t launch_dataflow_ty(const DfParams<T> &p, int nf, int lim, int grid, cudaStream_t s, int *grid_out);

template <typename T>
inline cudaError_t launch_dataflow(const DfParams<T> &p, int nf, int lim, int grid, cudaStream_t s, int *grid_out) {
    return launch_dataflow_ty<T, 8>(p, nf, lim, grid, s, grid_out);
}

}  // namespace asuca
