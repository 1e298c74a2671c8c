// Lateral and upper damping of the prognostic fields toward boundary data
// (Sec. 2.1: the damping kernel of the dynamical core that the paper uses as
// its parallel-loop example).  Per cell and field:
//   ptb_damp = mtratio (ref + bnd0) + tratio (ref + bnd1) - ref   (the paper's kernel:
//              the boundary perturbation interpolated in time between two datasets)
//   target   = ref + ptb_damp
//   y       <- (y + a target) / (1 + a),  a = dt nu(i, j, k)      (implicit Rayleigh relaxation)
// with nu = max(nu_lat w_lat, nu_top w_top), w_lat = ((width - d) / width)^2 for
// cells d < width cells from the nearest i or j edge, w_top = ((kk + 1) / ntop)^2
// on the kk-th of the top ntop levels, zero elsewhere.
//
// Only the damping zone is touched: the frame of `width` cells on every
// lateral side below the top zone, and the whole of the top ntop levels.  The
// zone's cells are enumerated by a flat index (level by level: the bottom
// rows, the top rows, then the left and right segments of the rows between;
// then the top levels plane by plane), so consecutive threads touch
// consecutive i and the grid is as large as the zone, not the domain.  The
// kernel streams 5F values per zone cell (ref, bnd0, bnd1, y in, y out); a =
// dt nu and the factors 1 / (1 + a), a / (1 + a) come from per-distance and
// per-level tables computed once on the host.  The target is used in its
// expanded form (the ref terms of ptb_damp and target cancel), which differs
// from the paper's order of operations by rounding only.
#include <algorithm>
#include <cstring>

#include "damping.cuh"

namespace asuca {

template <typename T>
struct DampParams {
    T *y[MAXF];
    const T *ref, *b0, *b1;   // [F][nz][ny][nx]
    size_t fs;                // field stride nz * nx * ny
    unsigned plane, frame, nlow, total;
    int nx, ny, nz, nf, width, ntop;
    T mt, tr;
    T a_lat[DAMP_MAXW], c_lat[DAMP_MAXW], ac_lat[DAMP_MAXW];
    T a_top[MAXNZ], c_top[MAXNZ], ac_top[MAXNZ];
};

template <typename T>
__global__ void __launch_bounds__(256) damping_kernel(const __grid_constant__ DampParams<T> p) {
    const unsigned W = (unsigned)p.width, nx = (unsigned)p.nx;
    for (unsigned u = blockIdx.x * blockDim.x + threadIdx.x; u < p.total; u += gridDim.x * blockDim.x) {
        unsigned i, j, k;
        damping_cell(u, W, nx, (unsigned)p.ny, (unsigned)p.nz, (unsigned)p.ntop, p.frame, p.nlow, p.plane, i, j, k);
        const int d = min(min((int)i, p.nx - 1 - (int)i), min((int)j, p.ny - 1 - (int)j));
        const int kk = (int)k - (p.nz - p.ntop);
        T a = T(0), c = T(1), ac = T(0);
        if (d < p.width) {
            a = p.a_lat[d];
            c = p.c_lat[d];
            ac = p.ac_lat[d];
        }
        if (kk >= 0 && p.a_top[kk] > a) {
            c = p.c_top[kk];
            ac = p.ac_top[kk];
        }
        // target = ref + ptb_damp = mtratio (ref + bnd0) + tratio (ref + bnd1), so
        // y' = c y + ac target = c y + (A + B) ref + A bnd0 + B bnd1 with
        // A = ac mtratio, B = ac tratio: four operations per field (the FP64
        // path is bound by the FP64 pipe otherwise)
        const T A = ac * p.mt, B = ac * p.tr, AB = A + B;
        const size_t o = (size_t)k * p.plane + (size_t)j * nx + i;
#pragma unroll 4
        for (int f = 0; f < p.nf; f++) {
            const size_t q = (size_t)f * p.fs + o;
            T *yf = p.y[f] + o;
            T v = c * *yf + AB * p.ref[q];
            v += A * p.b0[q];
            *yf = v + B * p.b1[q];
        }
    }
}

template <typename T>
cudaError_t launch_damping(T *const *y, int nf, const T *ref, const T *b0, const T *b1, int nx, int ny, int nz,
                           int width, int ntop, double nu_lat, double nu_top, double mtratio, double tratio,
                           double dt, int sms, cudaStream_t s) {
    DampParams<T> p;
    std::memset(&p, 0, sizeof(p));
    for (int f = 0; f < MAXF; f++) p.y[f] = f < nf ? y[f] : nullptr;
    p.ref = ref;
    p.b0 = b0;
    p.b1 = b1;
    const DampZone z = damping_zone(nx, ny, nz, width, ntop);
    p.plane = z.plane;
    p.fs = (size_t)p.plane * nz;
    p.frame = z.frame;
    p.nlow = z.nlow;
    p.total = z.total;
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    p.nf = nf;
    p.width = width;
    p.ntop = ntop;
    p.mt = (T)mtratio;
    p.tr = (T)tratio;
    // a = dt nu per distance from the edge and per top level, with the
    // implicit-relaxation factors 1 / (1 + a) and a / (1 + a)
    for (int d = 0; d < width; d++) {
        const double x = (double)(width - d) / width;
        const double a = dt * (nu_lat * (x * x));
        p.a_lat[d] = (T)a;
        p.c_lat[d] = (T)(1.0 / (1.0 + a));
        p.ac_lat[d] = (T)(a / (1.0 + a));
    }
    for (int kk = 0; kk < ntop; kk++) {
        const double x = (double)(kk + 1) / ntop;
        const double a = dt * (nu_top * (x * x));
        p.a_top[kk] = (T)a;
        p.c_top[kk] = (T)(1.0 / (1.0 + a));
        p.ac_top[kk] = (T)(a / (1.0 + a));
    }
    if (p.total == 0) return cudaSuccess;
    const unsigned want = (p.total + 255u) / 256u;
    const unsigned cap = (unsigned)std::max(sms, 1) * 8u;
    damping_kernel<T><<<std::min(want, cap), 256, 0, s>>>(p);
    return cudaGetLastError();
}

template cudaError_t launch_damping<float>(float *const *, int, const float *, const float *, const float *, int, int,
                                           int, int, int, double, double, double, double, double, int, cudaStream_t);
template cudaError_t launch_damping<double>(double *const *, int, const double *, const double *, const double *, int,
                                            int, int, int, int, double, double, double, double, double, int,
                                            cudaStream_t);

}  // namespace asuca
