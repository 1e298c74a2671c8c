// One explicit 7-point diffusion step, the kernel of the reduced weather
// application of Sec. 4 "Productivity- and Performance Results", in two
// storage orders with the same thread mapping, to measure what Sec. 1.3
// "Memory Layout" states: a GPU needs its first parallel dimension (here i,
// threadIdx.x) to be the stride-1 one.
//   IJK: element (i, j, k) at (k ny + j) nx + i   (i fastest)
//   KIJ: element (i, j, k) at (j nx + i) nz + k   (k fastest, the order ASUCA uses on CPU)
// out = in + c (sum of the six neighbours - 6 in), periodic in i and j, zero
// flux through the lids.  A thread owns a chunk of KC levels of an (i, j)
// column (grid z: the chunks) and marches them with the column's values at
// k-1, k, k+1 in registers; the four horizontal neighbours are loaded one
// level ahead (the caches supply their reuse).  Every address is the
// neighbour column's offset plus k times the level stride, so the two orders
// differ only in those two numbers.
#include "common.cuh"

namespace asuca {

constexpr int S7_KC = 16;   // levels per thread

template <typename T, int LAYOUT>
__global__ void __launch_bounds__(256) stencil7_kernel(const T *__restrict__ in, T *__restrict__ out, int nx, int ny,
                                                       int nz, T c) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const int k0 = blockIdx.z * S7_KC, k1 = min(k0 + S7_KC, nz);
    const int iw = i > 0 ? i - 1 : nx - 1, ie = i < nx - 1 ? i + 1 : 0;
    const int js = j > 0 ? j - 1 : ny - 1, jn = j < ny - 1 ? j + 1 : 0;
    // column offset of (ii, jj) and the stride between levels
    auto col = [&](int ii, int jj) -> size_t {
        return LAYOUT == 0 ? (size_t)jj * nx + ii : ((size_t)jj * nx + ii) * nz;
    };
    const size_t ls = LAYOUT == 0 ? (size_t)nx * ny : 1;
    const T *pc = in + col(i, j), *pw = in + col(iw, j), *pe = in + col(ie, j), *ps = in + col(i, js),
            *pn = in + col(i, jn);
    T *po = out + col(i, j);
    T mid = pc[k0 * ls];
    T below = k0 > 0 ? pc[(k0 - 1) * ls] : mid;   // the ghost under the bottom level copies it
    T w = pw[k0 * ls], e = pe[k0 * ls], so = ps[k0 * ls], no = pn[k0 * ls];
    for (int k = k0; k < k1; k++) {
        const size_t kn = (size_t)(k + 1 < nz ? k + 1 : k) * ls;
        const T above = pc[kn];
        const T w1 = pw[kn], e1 = pe[kn], s1 = ps[kn], n1 = pn[kn];
        const T sum = w + e + so + no + below + above;
        po[(size_t)k * ls] = mid + c * (sum - T(6) * mid);
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
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8, (nz + S7_KC - 1) / S7_KC);
    if (layout == 0) stencil7_kernel<T, 0><<<grid, block, 0, s>>>(in, out, nx, ny, nz, c);
    else stencil7_kernel<T, 1><<<grid, block, 0, s>>>(in, out, nx, ny, nz, c);
    return cudaGetLastError();
}

template cudaError_t launch_stencil7<float>(const float *, float *, int, int, int, int, float, cudaStream_t);
template cudaError_t launch_stencil7<double>(const double *, double *, int, int, int, int, double, cudaStream_t);

}  // namespace asuca
