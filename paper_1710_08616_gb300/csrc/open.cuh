// Kernels of the open lateral boundaries (open.cu): the stage-1 input of an
// open domain and the halo strips of its padded stage buffers.
#pragma once

#include "common.cuh"

namespace asuca {

template <typename T>
struct OpenParams {
    const T *y[MAXF];        // caller fields (rho, rho*phi), unpadded [nz][ny][nx]
    T *pad[MAXF];            // padded buffer: per-field views (pair layout; element (k, j, i) at
                             // k pplane + (j + 2) pitch + 2 (i + 4))
    const T *hin0, *hin1;    // halo-layout input: received strips / boundary data (hin1: second dataset or null)
    T *hout;                 // halo-layout output (pack)
    long long pitch, pplane; // the pair layout's row and level strides (elements)
    int nx, ny, nz, nt;      // nt = F - 1 transported fields
    T w0, w1;                // time weights of hin0, hin1 (1 - tratio, tratio)
};

// phi of every interior cell into the padded buffer (fields 1 .. F-1)
template <typename T>
cudaError_t launch_open_prepare(const OpenParams<T> &p, cudaStream_t s);
// pack: the block's edge strips into p.hout; unpack: p.hin0 (and p.hin1,
// weighted) into the ghost cells
template <typename T>
cudaError_t launch_halo(const OpenParams<T> &p, bool pack, int nsm, cudaStream_t s);

}  // namespace asuca
