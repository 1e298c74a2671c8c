// Launcher of the lateral and upper damping kernel (damping.cu).
#pragma once

#include "common.cuh"

namespace asuca {

constexpr int DAMP_MAXW = ASUCA_DAMP_MAX_WIDTH;

// The damping zone as a flat index u in [0, total): level by level below the
// top zone, the frame (width W) of the level: first the W bottom rows, then
// the W top rows, then the left and right W-cell segments of the rows
// between; after those (u >= nlow) the top ntop levels plane by plane.
// frame = 2 W nx + 2 W (ny - 2 W) cells per level, nlow = (nz - ntop) frame.
// Used by the kernel and, through asuca_debug_damping_cells, by host tests.
__host__ __device__ __forceinline__ void damping_cell(unsigned u, unsigned W, unsigned nx, unsigned ny, unsigned nz,
                                                      unsigned ntop, unsigned frame, unsigned nlow, unsigned plane,
                                                      unsigned &i, unsigned &j, unsigned &k) {
    if (u < nlow) {   // lateral frame of a level below the top zone
        k = u / frame;
        unsigned r = u - k * frame;
        const unsigned wn = W * nx;
        if (r < wn) {                       // bottom rows j < W
            j = r / nx;
            i = r - j * nx;
        } else if (r < 2 * wn) {            // top rows j >= ny - W
            r -= wn;
            const unsigned jj = r / nx;
            i = r - jj * nx;
            j = ny - W + jj;
        } else {                            // left and right segments of the rows between
            r -= 2 * wn;
            const unsigned jj = r / (2 * W), c = r - jj * (2 * W);
            j = W + jj;
            i = c < W ? c : nx - 2 * W + c;
        }
    } else {          // a whole level of the top zone
        const unsigned r = u - nlow;
        const unsigned kk = r / plane, c = r - kk * plane;
        k = nz - ntop + kk;
        j = c / nx;
        i = c - j * nx;
    }
}

// cells per level plane, frame cells per level, frame cells below the top
// zone, and all zone cells
struct DampZone {
    unsigned plane, frame, nlow, total;
};
inline DampZone damping_zone(int nx, int ny, int nz, int width, int ntop) {
    DampZone z;
    z.plane = (unsigned)nx * (unsigned)ny;
    z.frame = 2u * width * nx + (unsigned)(ny - 2 * width) * 2u * width;
    z.nlow = (unsigned)(nz - ntop) * z.frame;
    z.total = z.nlow + (unsigned)ntop * z.plane;
    return z;
}

// y[f] (nf fields of the state), ref/b0/b1 ([nf][nz][ny][nx]) on the device;
// the zone and rates as asuca_damping documents them, already validated.
template <typename T>
cudaError_t launch_damping(T *const *y, int nf, const T *ref, const T *b0, const T *b1, int nx, int ny, int nz,
                           int width, int ntop, double nu_lat, double nu_top, double mtratio, double tratio,
                           double dt, int sms, cudaStream_t s);

}  // namespace asuca
