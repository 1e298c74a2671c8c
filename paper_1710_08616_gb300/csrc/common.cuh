// Device-side building blocks shared by the stage and column kernels.
//
// Layout: every 3D field is [nz][ny][nx], i fastest (the IJK order of
// Sec. 1.3 "Memory Layout": the first parallel dimension is the stride-1
// dimension so that a warp's loads coalesce).  One thread owns one (i, j)
// column and marches k (Sec. 1.1: parallel in I/J, sequential in K).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "asuca.h"

namespace asuca {

constexpr int MAXF = 2 + ASUCA_MAX_TRACERS;   // rho, rho*theta, tracers
constexpr int MAXNZ = ASUCA_MAX_NZ;

// ------------------------------------------------------------------ params

template <typename T>
struct StageParams {
    const T *yin[MAXF];     // stage input Y^(s-1): phi and fluxes come from here
    const T *ybase[MAXF];   // Y^n
    T *yout[MAXF];          // Y^(s) = Y^n + cdt * R(Y^(s-1))
    const T *mu, *mv, *mw;
    const T *tend;          // [F-1][nz][ny][nx] or nullptr
    int nx, ny, nz, lim;
    long long plane;        // nx * ny
    T cdt, rdx, rdy;
    T rdz[MAXNZ];           // 1 / dz_k
};

template <typename T>
struct ColumnParams {
    T *y[MAXF];
    int nx, ny, nz, sed;    // sed: tracer field index (2 + n) or -1
    long long plane;
    int do_relax, do_sed, do_diff, do_phys, budgets;
    T relax_r;              // dt / tau
    T relax_inv;            // 1 / (1 + dt / tau)
    T sed_dt;               // dt
    T sed_v;                // fall speed
    double dt, dxdy;
    double *precip_col;     // [ny][nx], accumulated dt * P_bottom * dx * dy
    double *partials;       // [gridDim.x][F + 1] budget partials (sum over columns of sum_k f dz)
    double *scratch;        // [nz][F + 1][nslots]
    long long nslots;
    T dzT[MAXNZ];           // dz_k
    T sedr[MAXNZ];          // 1 / (dz_k + dt v)
    T thref[MAXNZ];         // theta_ref(z_k)
    double dz[MAXNZ];
    double kc[MAXNZ];       // dt K(z_{k+1/2}) / dzc_{k+1/2} / 2 for face k+1/2 (0 at the top lid)
    double dzr_up[MAXNZ];   // dz_{k+1} / dz_k
    double dzr_dn[MAXNZ];   // dz_{k-1} / dz_k
};

// ------------------------------------------------------------------ helpers

__host__ __device__ __forceinline__ int wrap_index(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// Reciprocal in double by Newton-Raphson iteration on f(y) = 1/y - x,
// y <- y (2 - x y), started from the hardware single-precision approximation.
// Each iteration squares the relative error: ~2^-22 -> ~2^-44 -> below 2^-53
// (the result is within a few ulp of 1/x).  Valid for |x| in the normal
// float range, which holds for densities and the diagonally dominant pivots
// of the vertical-diffusion solve.
__device__ __forceinline__ double rcp_newton(double x) {
    float xf = (float)x, yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(xf));
    double y = (double)yf;
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    return y;
}

template <typename T> __device__ __forceinline__ T recip(T x);
template <> __device__ __forceinline__ double recip<double>(double x) { return rcp_newton(x); }
template <> __device__ __forceinline__ float recip<float>(float x) { return __frcp_rn(x); }

// Koren limiter increment L(d0, d1) = psi(d1/d0) d0 in division-free form:
// sgn(d0) min(2|d1|, (|d0| + 2|d1|)/3, 2|d0|) when d0 and d1 share a sign,
// else 0.  If either is zero the min is zero, so only the sign test is needed.
template <typename T>
__device__ __forceinline__ T limiter(T d0, T d1, int lim) {
    if (lim == ASUCA_LIM_LINEAR) return (d0 + T(2) * d1) * T(1.0 / 3.0);
    if (lim == ASUCA_LIM_UPWIND1) return T(0);
    const T a0 = fabs(d0), a1 = fabs(d1);
    const T m = fmin(T(2) * a1, fmin((a0 + T(2) * a1) * T(1.0 / 3.0), T(2) * a0));
    return (signbit(d0) == signbit(d1)) ? copysign(m, d0) : T(0);
}

// Face value at i+1/2 from phi at i-1, i, i+1, i+2, upwind by the sign of the
// face mass flux m (m = 0 counts as m >= 0): the mirrored stencil for m < 0.
template <typename T>
__device__ __forceinline__ T face_value(T pm1, T p0, T p1, T p2, T m, int lim) {
    const bool up = m >= T(0);
    const T c = up ? p0 : p1;
    const T d0 = up ? (p0 - pm1) : (p1 - p2);
    const T d1 = up ? (p1 - p0) : (p0 - p1);
    return c + T(0.5) * limiter(d0, d1, lim);
}

// ------------------------------------------------------------------ launchers

template <typename T>
cudaError_t launch_stage(const StageParams<T> &p, int nf, cudaStream_t s);

template <typename T>
cudaError_t launch_column(const ColumnParams<T> &p, int nf, int grid, int block, cudaStream_t s);

cudaError_t launch_budget_reduce(const double *partials, int nblocks, int nq, int nf,
                                 double dxdy, double *out, int *status, cudaStream_t s);

constexpr int COL_TPB = 128;

}  // namespace asuca
