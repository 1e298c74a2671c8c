// One explicit 7-point diffusion step, the kernel of the reduced weather
// application of Sec. 4 "Productivity- and Performance Results", in two
// storage orders with the same thread mapping, to measure what Sec. 1.3
// "Memory Layout" states: a GPU needs its first parallel dimension (here i,
// threadIdx.x) to be the stride-1 one.
//   IJK: element (i, j, k) at (k ny + j) nx + i   (i fastest)
//   KIJ: element (i, j, k) at (j nx + i) nz + k   (k fastest, the order ASUCA uses on CPU)
// out = in + c (sum of the six neighbours - 6 in), periodic in i and j, zero
// flux through the lids.  A thread owns four consecutive cells in i of a row
// j and a chunk of KC levels (grid z: the chunks), and marches the chunk with
// the cells' values at k-1, k, k+1 in registers; the neighbouring rows' four
// cells and the two cells beyond the group's ends in i are loaded one level
// ahead (the caches supply their reuse).  Every address is a column's offset
// plus k times the level stride, so the two orders differ only in those two
// numbers; in IJK with nx a multiple of 4 the four cells of a row are one
// 16-byte access.  The arithmetic per cell is the same in both orders.
#include "common.cuh"

namespace asuca {

constexpr int S7_KC = 16;   // levels per thread
constexpr int S7_V = 4;     // consecutive cells in i per thread

template <typename T> __device__ __forceinline__ void ld_vec4(const T *p, T (&v)[S7_V]);
template <> __device__ __forceinline__ void ld_vec4<float>(const float *p, float (&v)[S7_V]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <> __device__ __forceinline__ void ld_vec4<double>(const double *p, double (&v)[S7_V]) {
    const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <typename T> __device__ __forceinline__ void st_vec4(T *p, const T (&v)[S7_V]);
template <> __device__ __forceinline__ void st_vec4<float>(float *p, const float (&v)[S7_V]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <> __device__ __forceinline__ void st_vec4<double>(double *p, const double (&v)[S7_V]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
}

// vec: IJK with nx a multiple of 4 and 16-byte aligned buffers (a group's
// four cells are one aligned vector)
template <typename T, int LAYOUT>
__global__ void __launch_bounds__(256) stencil7_kernel(const T *__restrict__ in, T *__restrict__ out, int nx, int ny,
                                                       int nz, T c, int vec) {
    const int i0 = (blockIdx.x * 32 + threadIdx.x) * S7_V, j = blockIdx.y * 8 + threadIdx.y;
    if (i0 >= nx || j >= ny) return;
    const int nv = min(S7_V, nx - i0);   // the group's cells inside the domain
    const bool vv = LAYOUT == 0 && vec && nv == S7_V;
    const int k0 = blockIdx.z * S7_KC, k1 = min(k0 + S7_KC, nz);
    const int iw = i0 > 0 ? i0 - 1 : nx - 1, ie = i0 + nv < nx ? i0 + nv : 0;   // beyond the group's ends
    const int js = j > 0 ? j - 1 : ny - 1, jn = j < ny - 1 ? j + 1 : 0;
    // column offset of (ii, jj) and the stride between levels
    auto col = [&](int ii, int jj) -> size_t {
        return LAYOUT == 0 ? (size_t)jj * nx + ii : ((size_t)jj * nx + ii) * nz;
    };
    const size_t ls = LAYOUT == 0 ? (size_t)nx * ny : 1;
    // the group's cells of row jj at level k
    auto row = [&](int jj, size_t kofs, T (&v)[S7_V]) {
        if (vv) {
            ld_vec4<T>(in + col(i0, jj) + kofs, v);
        } else {
#pragma unroll
            for (int q = 0; q < S7_V; q++) v[q] = q < nv ? in[col(i0 + q, jj) + kofs] : T(0);
        }
    };
    const size_t cw = col(iw, j), ce = col(ie, j);
    T mid[S7_V], below[S7_V], so[S7_V], no[S7_V];
    size_t kofs = (size_t)k0 * ls;
    row(j, kofs, mid);
    if (k0 > 0) row(j, kofs - ls, below);   // the ghost under the bottom level copies it
#pragma unroll
    for (int q = 0; q < S7_V; q++)
        if (k0 == 0) below[q] = mid[q];
    row(js, kofs, so);
    row(jn, kofs, no);
    T w = in[cw + kofs], e = in[ce + kofs];
    for (int k = k0; k < k1; k++) {
        const size_t kn = (size_t)(k + 1 < nz ? k + 1 : k) * ls;
        T above[S7_V], s1[S7_V], n1[S7_V];
        row(j, kn, above);
        row(js, kn, s1);
        row(jn, kn, n1);
        const T w1 = in[cw + kn], e1 = in[ce + kn];
        T o[S7_V];
#pragma unroll
        for (int q = 0; q < S7_V; q++) {
            const T wq = q == 0 ? w : mid[q - 1];
            const T eq = q == nv - 1 ? e : (q + 1 < S7_V ? mid[q + 1] : T(0));
            const T sum = wq + eq + so[q] + no[q] + below[q] + above[q];
            o[q] = mid[q] + c * (sum - T(6) * mid[q]);
        }
        const size_t ko = (size_t)k * ls;
        if (vv) {
            st_vec4<T>(out + col(i0, j) + ko, o);
        } else {
#pragma unroll
            for (int q = 0; q < S7_V; q++)
                if (q < nv) out[col(i0 + q, j) + ko] = o[q];
        }
#pragma unroll
        for (int q = 0; q < S7_V; q++) {
            below[q] = mid[q];
            mid[q] = above[q];
            so[q] = s1[q];
            no[q] = n1[q];
        }
        w = w1;
        e = e1;
    }
}

template <typename T>
cudaError_t launch_stencil7(const T *in, T *out, int nx, int ny, int nz, int layout, T c, cudaStream_t s) {
    const int vec = layout == 0 && nx % S7_V == 0 && (reinterpret_cast<uintptr_t>(in) % 16) == 0 &&
                    (reinterpret_cast<uintptr_t>(out) % 16) == 0;
    dim3 block(32, 8), grid((nx + 32 * S7_V - 1) / (32 * S7_V), (ny + 7) / 8, (nz + S7_KC - 1) / S7_KC);
    if (layout == 0) stencil7_kernel<T, 0><<<grid, block, 0, s>>>(in, out, nx, ny, nz, c, vec);
    else stencil7_kernel<T, 1><<<grid, block, 0, s>>>(in, out, nx, ny, nz, c, vec);
    return cudaGetLastError();
}

template cudaError_t launch_stencil7<float>(const float *, float *, int, int, int, int, float, cudaStream_t);
template cudaError_t launch_stencil7<double>(const double *, double *, int, int, int, int, double, cudaStream_t);

}  // namespace asuca
