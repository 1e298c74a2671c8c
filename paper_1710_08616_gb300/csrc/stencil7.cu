// One explicit 7-point diffusion step, the kernel of the reduced weather
// application of Sec. 4 "Productivity- and Performance Results", in two
// storage orders with the same thread mapping, to measure what Sec. 1.3
// "Memory Layout" states: a GPU needs its first parallel dimension (here i,
// threadIdx.x) to be the stride-1 one.
//   IJK: element (i, j, k) at (k ny + j) nx + i   (i fastest)
//   KIJ: element (i, j, k) at (j nx + i) nz + k   (k fastest, the order ASUCA uses on CPU)
// out = in + c (sum of the six neighbours - 6 in), periodic in i and j, zero
// flux through the lids.  A thread owns an (i, j) column and marches k with
// the column's values at k-1, k, k+1 in registers; the four horizontal
// neighbours are loaded at each level (the caches supply their reuse).
#include "common.cuh"

namespace asuca {

template <typename T, int LAYOUT>
__global__ void __launch_bounds__(256) stencil7_kernel(const T *__restrict__ in, T *__restrict__ out, int nx, int ny,
                                                       int nz, T c) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const int iw = i > 0 ? i - 1 : nx - 1, ie = i < nx - 1 ? i + 1 : 0;
    const int js = j > 0 ? j - 1 : ny - 1, jn = j < ny - 1 ? j + 1 : 0;
    auto at = [&](int ii, int jj, int k) -> size_t {
        return LAYOUT == 0 ? ((size_t)k * ny + jj) * nx + ii : ((size_t)jj * nx + ii) * nz + k;
    };
    T mid = in[at(i, j, 0)];
    T below = mid;   // the ghost under the bottom level copies it
    // the horizontal neighbours are loaded one level ahead
    T w = in[at(iw, j, 0)], e = in[at(ie, j, 0)], so = in[at(i, js, 0)], no = in[at(i, jn, 0)];
    for (int k = 0; k < nz; k++) {
        const int kn = k + 1 < nz ? k + 1 : k;
        const T above = in[at(i, j, kn)];
        const T w1 = in[at(iw, j, kn)], e1 = in[at(ie, j, kn)], s1 = in[at(i, js, kn)], n1 = in[at(i, jn, kn)];
        const T sum = w + e + so + no + below + above;
        out[at(i, j, k)] = mid + c * (sum - T(6) * mid);
        below = mid;
        mid = above;
        w = w1;
        e = e1;
        so = s1;
        no = n1;
    }
}

template <typename T>
cudaError_t launch_stencil7(const T *in, T *out, int nx, int ny, int nz, int layout, T c, cudaStream_t s) {
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8);
    if (layout == 0) stencil7_kernel<T, 0><<<grid, block, 0, s>>>(in, out, nx, ny, nz, c);
    else stencil7_kernel<T, 1><<<grid, block, 0, s>>>(in, out, nx, ny, nz, c);
    return cudaGetLastError();
}

template cudaError_t launch_stencil7<float>(const float *, float *, int, int, int, int, float, cudaStream_t);
template cudaError_t launch_stencil7<double>(const double *, double *, int, int, int, int, double, cudaStream_t);

}  // namespace asuca
