// Open (non-periodic) lateral boundaries: a limited-area domain fed by
// boundary data (the boundary datasets of the damping kernel, Sec. 2.1), or
// one block of a horizontally decomposed domain exchanging halos with its
// neighbours (Sec. 1.1: horizontal blocks with halo communication; Sec. 2.2:
// halo updates every time step).
//
// The stage kernel reads its lateral neighbours from the two ghost columns
// and rows of its padded input buffer (the pair layout of common.cuh, logical
// (i, j) at (i+4, j+2)); in the open mode nothing wraps and no stage writes
// those ghosts.  The kernels here fill and read them:
//   * open_prepare_kernel: the stage-1 input, phi = (rho phi) / rho of every
//     interior cell (one reciprocal of rho per cell, as the periodic stage-1
//     path converts), fields 1 .. F-1;
//   * halo_pack_kernel: the strips a block sends to its neighbours (its two
//     westmost columns to the west neighbour, and so on);
//   * halo_unpack_kernel: received strips (or boundary data, optionally
//     interpolated in time between two datasets) into the ghost cells.
// Halo layout (send and receive buffers, boundary data): four strips one
// after another, W, E ([F-1][nz][2][ny] each), S, N ([F-1][nz][2][nx] each).
// Packed, strip W holds cells i = c, E holds i = nx-2+c, S holds j = c, N
// holds j = ny-2+c (c = 0, 1); unpacked, strip W fills ghosts i = c-2, E
// fills i = nx+c, S fills j = c-2, N fills j = ny+c.  So the W strip a block
// receives is its west neighbour's packed E strip, and so on.
// The stencil never reads the ghost corners (its stencil is a cross), so no
// diagonal messages are needed.
#include "open.cuh"

namespace asuca {

// strip, field, level, c and position of halo element u
struct HaloPos {
    int strip, f, k, c, pos;
};
__device__ __forceinline__ HaloPos halo_pos(long long u, int nx, int ny, int nz, int nt) {
    const long long sw = (long long)nt * nz * 2 * ny, ss = (long long)nt * nz * 2 * nx;
    HaloPos h;
    long long r;
    int len;
    if (u < 2 * sw) {
        h.strip = u < sw ? 0 : 1;
        r = u - h.strip * sw;
        len = ny;
    } else {
        r = u - 2 * sw;
        h.strip = r < ss ? 2 : 3;
        r -= (h.strip - 2) * ss;
        len = nx;
    }
    h.pos = (int)(r % len);
    r /= len;
    h.c = (int)(r % 2);
    r /= 2;
    h.k = (int)(r % nz);
    h.f = (int)(r / nz);
    return h;
}

template <typename T>
__global__ void open_prepare_kernel(const __grid_constant__ OpenParams<T> p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int k = blockIdx.z;
    if (i >= p.nx) return;
    const size_t o = ((size_t)k * p.ny + j) * p.nx + i;
    const size_t po = (size_t)k * p.pplane + (size_t)(j + 2) * p.pitch + 2 * (i + 4);
    const T r = recip(p.y[0][o]);
    for (int f = 1; f <= p.nt; f++) p.pad[f][po] = p.y[f][o] * r;
}

template <typename T>
__global__ void halo_pack_kernel(const __grid_constant__ OpenParams<T> p, long long total) {
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += (long long)gridDim.x * blockDim.x) {
        const HaloPos h = halo_pos(u, p.nx, p.ny, p.nz, p.nt);
        int i, j;
        if (h.strip < 2) {
            j = h.pos;
            i = h.strip == 0 ? h.c : p.nx - 2 + h.c;
        } else {
            i = h.pos;
            j = h.strip == 2 ? h.c : p.ny - 2 + h.c;
        }
        p.hout[u] = p.pad[1 + h.f][(size_t)h.k * p.pplane + (size_t)(j + 2) * p.pitch + 2 * (i + 4)];
    }
}

template <typename T>
__global__ void halo_unpack_kernel(const __grid_constant__ OpenParams<T> p, long long total) {
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += (long long)gridDim.x * blockDim.x) {
        const HaloPos h = halo_pos(u, p.nx, p.ny, p.nz, p.nt);
        int i, j;
        if (h.strip < 2) {
            j = h.pos;
            i = h.strip == 0 ? h.c - 2 : p.nx + h.c;
        } else {
            i = h.pos;
            j = h.strip == 2 ? h.c - 2 : p.ny + h.c;
        }
        T v = p.hin0[u];
        if (p.hin1) v = p.w0 * v + p.w1 * p.hin1[u];
        p.pad[1 + h.f][(size_t)h.k * p.pplane + (size_t)(j + 2) * p.pitch + 2 * (i + 4)] = v;
    }
}

template <typename T>
cudaError_t launch_open_prepare(const OpenParams<T> &p, cudaStream_t s) {
    dim3 block(128), grid((p.nx + 127) / 128, p.ny, p.nz);
    open_prepare_kernel<T><<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_halo(const OpenParams<T> &p, bool pack, int nsm, cudaStream_t s) {
    const long long total = (long long)p.nt * p.nz * 2 * (2LL * p.nx + 2LL * p.ny);
    if (total == 0) return cudaSuccess;
    const long long want = (total + 255) / 256, cap = (long long)nsm * 8;
    const int grid = (int)(want < cap ? want : cap);
    if (pack) halo_pack_kernel<T><<<grid, 256, 0, s>>>(p, total);
    else halo_unpack_kernel<T><<<grid, 256, 0, s>>>(p, total);
    return cudaGetLastError();
}

template cudaError_t launch_open_prepare<float>(const OpenParams<float> &, cudaStream_t);
template cudaError_t launch_open_prepare<double>(const OpenParams<double> &, cudaStream_t);
template cudaError_t launch_halo<float>(const OpenParams<float> &, bool, int, cudaStream_t);
template cudaError_t launch_halo<double>(const OpenParams<double> &, bool, int, cudaStream_t);

}  // namespace asuca
