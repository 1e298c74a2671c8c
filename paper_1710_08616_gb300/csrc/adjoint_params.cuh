// Parameters and launchers of the adjoint kernels (adjoint.cu).
#pragma once

#include "common.cuh"

namespace asuca {

template <typename T>
struct AdjStageParams {
    const T *ys[MAXF];            // stage input Y (element (k,j,i) at k*ys_plane + (j+ys_oy)*ys_pitch + (i+ys_ox)*ys_xs)
    long long ys_pitch, ys_plane;
    int ys_ox, ys_oy, ys_xs;
    int ys_phi;                   // 1: fields 1.. of ys hold phi (padded stage buffers); 0: rho*phi
    const T *lam[MAXF];           // adjoint of the stage output, [nz][ny][nx]
    T cs;                         // c_s * dt
    const uint8_t *branch;        // [F-1][nz][ny][nx], recorded by the forward stage
    const T *facev;               // [3][F-1][nz][ny][nx] face values of each cell's +1/2 faces, recorded too
    const T *mu, *mv, *mw;
    T *out1[MAXF];                // if set: R_Y^T (cs lam)
    T *out2[MAXF];                // if set: base2 + R_Y^T (cs lam) (+ lam if add_self)
    const T *base2[MAXF];
    int add_self;
    T *gmu, *gmv, *gmw;           // += R_M^T (cs lam)
    int nx, ny, nz;
    long long plane;
    T rdx, rdy;
    T rdz[MAXNZ];
};

template <typename T>
struct AdjColParams {
    ColumnParams<T> c;            // physics constants of the forward column pass (c.y = state before it)
    T *lam[MAXF];                 // in: adjoint of the column output; out: adjoint of its input
};

template <typename T>
cudaError_t launch_adj_stage(const AdjStageParams<T> &p, int nf, int lim, cudaStream_t s);

template <typename T>
cudaError_t launch_adj_column(const AdjColParams<T> &p, int nf, int grid, cudaStream_t s);

}  // namespace asuca
