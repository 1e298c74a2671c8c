// Device-side building blocks shared by the stage and column kernels.
//
// Layout: every 3D field is [nz][ny][nx], i fastest (the IJK order of
// Sec. 1.3 "Memory Layout": the first parallel dimension is the stride-1
// dimension so that a warp's loads coalesce).  One thread owns one (i, j)
// column and marches k (Sec. 1.1: parallel in I/J, sequential in K).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "asuca.h"

namespace asuca {

constexpr int MAXF = 2 + ASUCA_MAX_TRACERS;   // rho, rho*theta, tracers
constexpr int MAXNZ = ASUCA_MAX_NZ;

// ------------------------------------------------------------------ params

// Tile, ring depth and shared-memory layout of the stage kernel.  A CTA is
// 32 x TY columns (one warp per row); a ring slot holds one level plane of the
// tile with a 4-column halo in i (2 used; the TMA box must start on a 16-byte
// boundary) and a 2-row halo in j, in one of two layouts:
//   raw (the caller's fields, stage 1): [F][SY][SX], every field a plane;
//   pair (the library's padded stage buffers): [SY][NPF][SX][2], the phi
//     fields in pairs (1, 2), (3, 4), ... with a pair's two values of a cell
//     side by side, so one 2-element load fetches both operands of a packed
//     operation.
template <typename T, int NF, int TYV = 8>
struct StageShape {
    static constexpr int TX = 32;
    static constexpr int TY = TYV;                       // tile rows: 4, 8 or 16 (an autotuned choice)
    static constexpr int D = 5;                          // ring depth (levels in flight + window)
    // CTAs resident per SM (shared memory and registers allow this many)
    static constexpr int MIN_BLOCKS = sizeof(T) == 8 ? 1 : (TYV >= 16 ? 1 : (TYV >= 8 ? 2 : 3));
    static constexpr int SX = TX + 8;
    static constexpr int SY = TY + 4;
    static constexpr int NT = NF - 1;                    // transported fields (phi)
    static constexpr int NPF = (NT + 1) / 2;             // pairs holding them
    static constexpr int SLOT_RAW = NF * SY * SX;        // >= 2 NPF SY SX, the pair layout's slot
    static constexpr int SLOT_ELEMS = (SLOT_RAW * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T);
    static constexpr unsigned TX_BYTES = (unsigned)(SLOT_RAW * sizeof(T));
    // a padded stage input lands its phi pairs only: the stencil never reads
    // the density, whose update depends on M alone
    static constexpr unsigned TX_BYTES_PAIR = (unsigned)(2 * NPF * SY * SX * sizeof(T));
    static constexpr size_t RING_BYTES = (size_t)D * SLOT_ELEMS * sizeof(T);
    // j-face fluxes of the tile's rows and the row below, and the i0-1/2 face
    // fluxes of its rows, both per pair ([NPF][TY+1][TX], [NPF][TY] of pairs)
    static constexpr size_t YS_BYTES = ((size_t)NPF * (TY + 1) * TX * 2 * sizeof(T) + 15) / 16 * 16;
    static constexpr size_t XB_BYTES = ((size_t)NPF * TY * 2 * sizeof(T) + 15) / 16 * 16;
    static constexpr size_t SMEM_BYTES = RING_BYTES + YS_BYTES + XB_BYTES + (size_t)D * 8;
};

// Padded layout of the library's own stage buffers (the inputs of stages 2
// and 3), pitch = nx + 8 rounded up to 8 elements, logical (i, j) at
// (i + 4, j + 2), the 2-wide periodic ghosts written by the producing stage:
// the F fields in NP = ceil(F / 2) pairs, in the order 1, 2, ..., F-1, 0
// (phi of theta and the tracers, then the density), each pair's two values
// of a cell side by side:
//   element of field f at ((k (ny + 4) + j + 2) NP + q) 2 pitch + 2 (i + 4) + lane,
//   q = pos / 2, lane = pos % 2, pos = f - 1 (f >= 1) or F - 1 (f = 0).
__host__ __device__ __forceinline__ long long padded_pitch(int nx) { return ((long long)nx + 8 + 7) / 8 * 8; }
__host__ __device__ __forceinline__ int pair_count(int nf) { return (nf + 1) / 2; }
__host__ __device__ __forceinline__ int pair_pos(int f, int nf) { return f == 0 ? nf - 1 : f - 1; }

template <typename T>
struct StageParams {
    CUtensorMap tmap;       // padded stage input (phi; rho in field 0), when tma_in
    CUtensorMap umap[3];    // caller's unpadded rho, rho*theta, rho*q (3D, 3D, 4D), when user_tma
    const T *yin[MAXF];     // unpadded stage input (rho, rho*phi), when !tma_in
    const T *ybase[MAXF];   // Y^n (unpadded)
    T *yout[MAXF];          // Y^(s) = Y^n + cdt * R(Y^(s-1)); for a padded output the per-field views of
                            // the buffer (pair layout), yout[1] (field 1: pair 0, lane 0) its base
    const T *mu, *mv, *mw;
    const T *tend;          // [F-1][nz][ny][nx] or nullptr
    int *status;            // device status word (mapped host memory)
    int nx, ny, nz, lim;
    int tma_in;             // input is a padded stage buffer holding phi (TMA)
    int out_padded;         // output to a padded stage buffer: phi for f >= 1 and rho, with periodic ghosts
    int user_tma;           // unpadded input through umap for tiles whose halo lies inside the domain
    int ty;                 // tile rows of the instantiation to launch (the TMA box height follows it)
    int open;               // open lateral boundaries: the padded input's ghost columns/rows hold the
                            // lateral neighbours (a halo exchange or boundary data wrote them), nothing
                            // wraps, the output's ghosts are not written, and mu, mv are the open
                            // domain's face fluxes [nz][ny][nx+1] (face i-1/2 at i) and [nz][ny+1][nx]
    long long plane_u, plane_v;   // level strides of mu and mv (the plane, or its open-domain sizes)
    uint8_t *branch;        // when recording: [F-1][nz][ny][nx] branch bytes (2 bits per direction)
    T *facev;               // when recording, if set: [3][F-1][nz][ny][nx] face values of the cell's
                            // i+1/2, j+1/2 and k+1/2 faces (k+1/2 of the top level: 0)
    long long plane;        // nx * ny
    long long opitch, oplane;   // padded buffers: pitch, and level stride (elements) of one field plane
    long long prow, plev;       // padded output: row and level strides of the pair layout (elements)
    T cdt, rdx, rdy;
    T hcdt;                 // a hook with own_rho: the density it receives is Y^n + hcdt R (the step's: dt)
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
    double *alpha;          // the fused column pass split over stages 2 and 3: [nz][plane] alpha of each level
    int *status;            // device status word (the bounds-check build records out-of-range indices)
    double *rec;            // if set: [nz][F + 2][plane] record of the diffusion solve for the adjoint:
                            // m, alpha, gamma of each level and the scaled solution z of each field
    T dzT[MAXNZ];           // dz_k (rounded to T)
    float dzlo[MAXNZ];      // dz_k - (float)dz_k, the low part for float budget sums
    T sedr[MAXNZ];          // 1 / (dz_k + dt v)
    T thref[MAXNZ];         // theta_ref(z_k)
    double dz[MAXNZ];
    double kc[MAXNZ];       // dt K(z_{k+1/2}) / dzc_{k+1/2} / 2 for face k+1/2 (0 at the top lid)
    double dzr_up[MAXNZ];   // dz_{k+1} / dz_k
    double dzr_dn[MAXNZ];   // dz_{k-1} / dz_k
    double rdz64[MAXNZ];    // 1 / dz_k
    T rdzT[MAXNZ];          // 1 / dz_k (rounded to T)
    T kcT[MAXNZ];           // kc rounded to T
};

// ------------------------------------------------------------------ bounds-check build

// With ASUCA_BOUNDS_CHECK every instrumented index is tested against its
// buffer's extent before the access: an index outside [0, n) records
// ASUCA_ERR_BOUNDS in the status word and is replaced by 0, so the access
// stays inside the buffer and the kernel carries on (no trap).  Without it
// ASUCA_BC expands to nothing.
#ifdef ASUCA_BOUNDS_CHECK
template <typename I>
__device__ __forceinline__ I bc_index(I idx, long long n, int *status) {
    if ((long long)idx >= 0 && (long long)idx < n) return idx;
    if (status) atomicCAS(status, 0, (int)ASUCA_ERR_BOUNDS);
    return I(0);
}
#define ASUCA_BC(idx, n, status) ((idx) = bc_index((idx), (long long)(n), (status)))
#else
#define ASUCA_BC(idx, n, status) ((void)0)
#endif

// ------------------------------------------------------------------ helpers

__host__ __device__ __forceinline__ int wrap_index(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// ---- float <-> double on the integer pipe -------------------------------
// On this GPU the hardware conversions between float and double issue on the
// FP64 pipe (1/64 of the FP32 rate), so the column solve converts through the
// IEEE-754 bit fields instead (binary32: 1+8+23 bits, bias 127; binary64:
// 1+11+52 bits, bias 1023).  Zero, subnormal, infinite and NaN inputs take
// the hardware path, so every result equals the hardware conversion.

// The rare inputs go to the hardware conversions in functions of their own,
// so that they are reached by a branch: a conversion the compiler predicated
// off would still take an issue slot of the FP64 pipe for every call.
static __device__ __noinline__ double f2d_hw(float x) { return (double)x; }
static __device__ __noinline__ float d2f_hw(double x) { return __double2float_rn(x); }

// Exact widening: exponent rebiased by 1023 - 127 = 896, mantissa shifted by 29.
__device__ __forceinline__ double f2d_bits(float x) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t e = u & 0x7f800000u;
    if (e == 0u || e == 0x7f800000u) return f2d_hw(x);
    const uint32_t hi = (u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + (896u << 20));
    return __hiloint2double((int)hi, (int)(u << 29));
}

// Narrowing with round-to-nearest-even on the 29 dropped mantissa bits; the
// rounding carry may ripple into the exponent (and to infinity above FLT_MAX),
// as IEEE rounding does.  Doubles outside the float normal range take the
// hardware path.
__device__ __forceinline__ float d2f_bits(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t ea = (hi >> 20) & 0x7ffu;
    if (ea < 897u || ea > 1150u) return d2f_hw(x);
    uint32_t mag = (((hi & 0x7fffffffu) - (896u << 20)) << 3) | (lo >> 29);
    const uint32_t rem = lo & 0x1fffffffu;
    mag += (rem > 0x10000000u || (rem == 0x10000000u && (mag & 1u))) ? 1u : 0u;
    return __uint_as_float((hi & 0x80000000u) | mag);
}

// Narrowing without a branch, for the values a column level converts
// together: exact for doubles in the float normal range (d2f_bits's bit
// path); ok is cleared otherwise, and the caller then converts the whole level
// again with d2f_bits (one branch per level instead of one per value).
__device__ __forceinline__ float d2f_fast(double x, bool &ok) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t ea = (hi >> 20) & 0x7ffu;
    ok = ok && (ea - 897u) < 254u;   // d2f_bits's bit path: ea in [897, 1150]
    uint32_t mag = (((hi & 0x7fffffffu) - (896u << 20)) << 3) | (lo >> 29);
    const uint32_t rem = lo & 0x1fffffffu;
    mag += (rem > 0x10000000u || (rem == 0x10000000u && (mag & 1u))) ? 1u : 0u;
    return __uint_as_float((hi & 0x80000000u) | mag);
}

// Widening of any float (zero, subnormal, inf, NaN included), for values that
// are only stored: the bit path, else the hardware conversion.
__device__ __forceinline__ double f2d_bits_any(float x) { return f2d_bits(x); }

template <typename T> __device__ __forceinline__ double to_f64(T x);
template <> __device__ __forceinline__ double to_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ double to_f64<float>(float x) { return f2d_bits(x); }
template <typename T> __device__ __forceinline__ T from_f64(double x);
template <> __device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_f64<float>(double x) { return d2f_bits(x); }

// Reciprocal in double from a float seed and one third-order correction.
// The seed y0 is the float reciprocal (rcp.approx, relative error below
// 2^-22 with the truncated operand) of x's leading 23 mantissa bits, built
// and widened on the integer pipe.  With e = 1 - x y0 (exact to rounding by
// FMA), 1/x = y0 / (1 - e) = y0 (1 + e + e^2 + e^3 + ...), so
// y = y0 + y0 (e + e^2) leaves a truncation error of order e^3 < 2^-66: the
// result is within an ulp of 1/x after three FP64 FMAs (the FP64 pipe bounds
// the column solve).  Valid for normal, finite, non-zero x whose magnitude
// lies in the float normal range (densities and the diagonally dominant
// pivots of the solve).
__device__ __forceinline__ double rcp_f64(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    // binary64 -> binary32 by truncation: exponent rebiased by 896, 20 + 3 mantissa bits
    const uint32_t xf = (hi & 0x80000000u) | ((((hi & 0x7fffffffu) - (896u << 20)) << 3) | (lo >> 29));
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__uint_as_float(xf)));
    const uint32_t u = __float_as_uint(rf);
    const double y0 = __hiloint2double((int)((u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + (896u << 20))),
                                       (int)(u << 29));
    const double e = fma(-x, y0, 1.0);
    return fma(y0, fma(e, e, e), y0);
}

template <typename T> __device__ __forceinline__ T recip(T x);
template <> __device__ __forceinline__ double recip<double>(double x) { return rcp_f64(x); }
template <> __device__ __forceinline__ float recip<float>(float x) { return __frcp_rn(x); }

// v with its sign flipped when s has its sign bit set (v * sgn(s) as a bit operation)
__device__ __forceinline__ float sign_transfer(float v, float s) {
    return __uint_as_float(__float_as_uint(v) ^ (__float_as_uint(s) & 0x80000000u));
}
__device__ __forceinline__ double sign_transfer(double v, double s) {
    return __longlong_as_double(__double_as_longlong(v) ^
                                (__double_as_longlong(s) & (long long)0x8000000000000000ull));
}

// Face value from the upwind cell c, the downwind cell o and the far upwind
// cell far, with the limiter fixed at compile time (for M >= 0 at face
// i+1/2: c = phi_i, o = phi_{i+1}, far = phi_{i-1}; for M < 0 the mirror:
// phi_{i+1}, phi_i, phi_{i+2}; M = 0 counts as M >= 0).  With d0 = c - far
// and d1 = o - c the face value is c + L(d0, d1) / 2 in either direction.
// Koren's increment L = sgn(d0) min(2|d1|, (|d0| + 2|d1|)/3, 2|d0|) when d0
// and d1 share a sign, else 0, is evaluated halved and division-free: with
// x = d1 carrying the sign it has relative to d0 (x >= 0 iff they share a
// sign) and a = |d0|,
//   L / 2 = sgn(d0) max(0, min(x, a, x/3 + a/6)).
// The caller picks the three cells by address, so nothing here depends on
// the flow direction.
// min(|a|, |b|) carrying the sign sgn(a) sgn(b) (one instruction: PTX
// min.xorsign.abs): non-negative exactly when a and b share a sign (or one of
// them is zero, where the magnitude is 0).
__device__ __forceinline__ float min_xorsign_abs(float a, float b) {
    float d;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

template <int LIM, typename T>
__device__ __forceinline__ T face_val(T c, T o, T far) {
    if (LIM == ASUCA_LIM_UPWIND1) return c;
    const T d1 = o - c;
    const T d0 = c - far;
    if (LIM == ASUCA_LIM_LINEAR) return c + fma(d1, T(1.0 / 3.0), d0 * T(1.0 / 6.0));
    if constexpr (std::is_same<T, float>::value) {
        // The same value in fewer instructions: u = sgn(d0 d1) min(|d0|, |d1|)
        // equals min(x, a) when d0 and d1 share a sign and is <= 0 otherwise,
        // and |d1/3 + d0/6| equals t when they share a sign (round-to-nearest is
        // symmetric in sign, so the rounding is the same); the outer max gives 0
        // for opposite signs either way.
        const float u = min_xorsign_abs(d1, d0);
        const float t = fabsf(fmaf(d1, 1.f / 3.f, d0 * (1.f / 6.f)));
        return c + copysignf(fmaxf(fminf(u, t), 0.f), d0);
    }
    const T x = sign_transfer(d1, d0);
    const T a = fabs(d0);
    const T t = fma(x, T(1.0 / 3.0), a * T(1.0 / 6.0));
    T h;
    if constexpr (std::is_same<T, double>::value) {
        // For x > 0, x, a and t are non-negative doubles, whose order is the
        // order of their bit patterns read as integers, so the minimum is taken
        // on the integer pipe (the FP64 pipe bounds the double path); x <= 0
        // gives 0.  Equal to max(0, min(x, a, t)) for every non-NaN input.
        const long long xi = __double_as_longlong(x), ai = __double_as_longlong(a), ti = __double_as_longlong(t);
        long long mi = xi < ai ? xi : ai;
        mi = mi < ti ? mi : ti;
        h = xi > 0 ? __longlong_as_double(mi) : 0.0;
    } else {
        h = fmax(fmin(fmin(x, a), t), T(0));
    }
    return c + copysign(h, d0);
}

// The same face value, also returning the limiter branch taken: 0 zero,
// 1 "2r", 2 "kappa=1/3", 3 "cap 2" (a tie keeps the earlier branch).  The
// adjoint differentiates each face along the branch its forward pass took.
template <int LIM, typename T>
__device__ __forceinline__ T face_val_br(T c, T o, T far, int &br) {
    if (LIM == ASUCA_LIM_UPWIND1) {
        br = 0;
        return c;
    }
    const T d1 = o - c;
    const T d0 = c - far;
    if (LIM == ASUCA_LIM_LINEAR) {
        br = 2;
        return c + fma(d1, T(1.0 / 3.0), d0 * T(1.0 / 6.0));
    }
    const T x = sign_transfer(d1, d0);
    const T a = fabs(d0);
    const T t2 = fma(x, T(1.0 / 3.0), a * T(1.0 / 6.0));
    T h = x;
    br = 1;
    if constexpr (std::is_same<T, double>::value) {
        // the comparisons on the integer pipe, as in face_val: for x > 0 the
        // operands are non-negative doubles, ordered as their bit patterns
        const long long xi = __double_as_longlong(x), ai = __double_as_longlong(a), ti = __double_as_longlong(t2);
        long long hi = xi;
        if (ti < hi) { hi = ti; br = 2; }
        if (ai < hi) { hi = ai; br = 3; }
        h = __longlong_as_double(hi);
        if (!(xi > 0 && ai > 0)) { h = T(0); br = 0; }
    } else {
        if (t2 < h) { h = t2; br = 2; }
        if (a < h) { h = a; br = 3; }
        if (!(x > T(0) && a > T(0))) { h = T(0); br = 0; }
    }
    return c + copysign(h, d0);
}

// Flux M * face through a face (cells as for face_val).
template <int LIM, typename T>
__device__ __forceinline__ T face_flux(T c, T o, T far, T m) { return m * face_val<LIM>(c, o, far); }
template <int LIM, typename T>
__device__ __forceinline__ T face_flux_br(T c, T o, T far, T m, int &br) { return m * face_val_br<LIM>(c, o, far, br); }

// Two fields' fluxes through the same face at once (fields f and f+1 in the
// two lanes of a float2), with the packed FP32x2 FMA/ADD/MUL of this GPU;
// every packed operation rounds as its scalar twin in face_val, so the result
// is bit-identical to two calls of face_flux.  Differences are taken as
// fma(b, -1, a) = a - b exactly.
template <int LIM>
__device__ __forceinline__ float2 face_flux2(float2 c, float2 o, float2 far, float m) {
    const float2 m2 = make_float2(m, m);
    if (LIM == ASUCA_LIM_UPWIND1) return __fmul2_rn(m2, c);
    const float2 neg1 = make_float2(-1.f, -1.f);
    const float2 d1 = __ffma2_rn(c, neg1, o);
    const float2 d0 = __ffma2_rn(far, neg1, c);
    if (LIM == ASUCA_LIM_LINEAR) {
        const float2 t = __ffma2_rn(d1, make_float2(1.f / 3.f, 1.f / 3.f), __fmul2_rn(d0, make_float2(1.f / 6.f, 1.f / 6.f)));
        return __fmul2_rn(m2, __fadd2_rn(c, t));
    }
    // the min.xorsign.abs form of face_val<float> (the same value)
    const float2 t = __ffma2_rn(d1, make_float2(1.f / 3.f, 1.f / 3.f), __fmul2_rn(d0, make_float2(1.f / 6.f, 1.f / 6.f)));
    const float hx = fmaxf(fminf(min_xorsign_abs(d1.x, d0.x), fabsf(t.x)), 0.f);
    const float hy = fmaxf(fminf(min_xorsign_abs(d1.y, d0.y), fabsf(t.y)), 0.f);
    return __fmul2_rn(m2, __fadd2_rn(c, make_float2(copysignf(hx, d0.x), copysignf(hy, d0.y))));
}

// Two fields' face values with their limiter branches (as face_val_br, whose
// value it equals bit for bit); times M they equal face_flux2's fluxes.
template <int LIM>
__device__ __forceinline__ float2 face_val2_br(float2 c, float2 o, float2 far, int2 &br) {
    if (LIM == ASUCA_LIM_UPWIND1) {
        br = make_int2(0, 0);
        return c;
    }
    const float2 neg1 = make_float2(-1.f, -1.f);
    const float2 d1 = __ffma2_rn(c, neg1, o);
    const float2 d0 = __ffma2_rn(far, neg1, c);
    if (LIM == ASUCA_LIM_LINEAR) {
        br = make_int2(2, 2);
        const float2 t = __ffma2_rn(d1, make_float2(1.f / 3.f, 1.f / 3.f), __fmul2_rn(d0, make_float2(1.f / 6.f, 1.f / 6.f)));
        return __fadd2_rn(c, t);
    }
    const float2 x = make_float2(sign_transfer(d1.x, d0.x), sign_transfer(d1.y, d0.y));
    const float2 a = make_float2(fabsf(d0.x), fabsf(d0.y));
    const float2 t = __ffma2_rn(x, make_float2(1.f / 3.f, 1.f / 3.f), __fmul2_rn(a, make_float2(1.f / 6.f, 1.f / 6.f)));
    auto pick = [](float xv, float av, float tv, int &b) {
        float h = xv;
        b = 1;
        if (tv < h) { h = tv; b = 2; }
        if (av < h) { h = av; b = 3; }
        if (!(xv > 0.f && av > 0.f)) { h = 0.f; b = 0; }
        return h;
    };
    const float hx = pick(x.x, a.x, t.x, br.x);
    const float hy = pick(x.y, a.y, t.y, br.y);
    return __fadd2_rn(c, make_float2(copysignf(hx, d0.x), copysignf(hy, d0.y)));
}

// Face value at i+1/2 from the four cells i-1 .. i+2 and the upwind predicate u = (M >= 0).
template <int LIM, typename T>
__device__ __forceinline__ T face_val4(T pm1, T p0, T p1, T p2, bool u) {
    return u ? face_val<LIM>(p0, p1, pm1) : face_val<LIM>(p1, p0, p2);
}

// d face / d phi at the stencil cells (pm1, p0, p1, p2) for upwind predicate u
// and branch br, whose increment is L = a d0 + b d1 with (a, b) = (0, 0),
// (0, 2), (1/3, 2/3), (2, 0):  u: face = p0 + (a (p0 - pm1) + b (p1 - p0)) / 2,
// !u: face = p1 + (a (p1 - p2) + b (p0 - p1)) / 2.
template <typename T>
__device__ __forceinline__ T face_coef(bool u, int br, int q) {
    const T a = br == 2 ? T(1.0 / 3.0) : (br == 3 ? T(2) : T(0));
    const T b = br == 1 ? T(2) : (br == 2 ? T(2.0 / 3.0) : T(0));
    const T up = T(1) + T(0.5) * a - T(0.5) * b;
    if (u) return q == 0 ? T(-0.5) * a : (q == 1 ? up : (q == 2 ? T(0.5) * b : T(0)));
    return q == 0 ? T(0) : (q == 1 ? T(0.5) * b : (q == 2 ? up : T(-0.5) * a));
}

// ------------------------------------------------------------------ launchers

template <typename T>
cudaError_t launch_stage(const StageParams<T> &p, int nf, cudaStream_t s);

// Encode the TMA descriptor of a padded stage buffer (F fields at base, pair
// layout) for tiles of ty rows: the phi pairs only.
template <typename T>
cudaError_t encode_stage_map(CUtensorMap *map, void *base, int nf, int nx, int ny, int nz, int ty);
// Tensor maps over the caller's unpadded rho, rho*theta and rho*q (N fields)
// with the stage box (40 x (ty + 4) x 1 [x N]); the caller checks that every
// base is 16-byte aligned and that a row (nx elements) is a multiple of 16 bytes.
template <typename T>
cudaError_t encode_user_maps(CUtensorMap *maps, const void *rho, const void *rhotheta, const void *rhoq, int ntr,
                             int nx, int ny, int nz, int ty);

// the stage kernels of one tile height (one translation unit each)
template <typename T, int TY>
cudaError_t launch_stage_ty(const StageParams<T> &p, int nf, cudaStream_t s);

template <typename T>
cudaError_t launch_column(const ColumnParams<T> &p, int nf, int grid, int block, cudaStream_t s);

// Stage 3 with the top-down half of the column pass (downward march), and
// the bottom-up half (fused_impl.cuh, column.cu).
template <typename T>
struct FusedParams {
    StageParams<T> s;       // stage 3: padded phi input (TMA), unpadded output
    ColumnParams<T> c;      // column constants; scratch is the fused scratch (fscratch_level layout), alpha
                            // the [nz][plane] array of the split column pass
};
template <typename T>
cudaError_t launch_stage3_column(const FusedParams<T> &p, int nf, cudaStream_t s);
// The fused column pass split over two stages: stage 2 (padded output, as
// launch_stage) with the FP64 factorisation into p.c.scratch and p.c.alpha,
// then stage 3 with the relaxation, sedimentation and elimination sweep.
template <typename T>
cudaError_t launch_stage2_factor(const FusedParams<T> &p, int nf, cudaStream_t s);
template <typename T>
cudaError_t launch_stage3_sweep(const FusedParams<T> &p, int nf, cudaStream_t s);

// Scratch of the fused column pass (ColDownHook writes it, column_up_kernel
// reads it): per level, the columns in groups of 32, each group's F + 1
// quantities as 32 consecutive doubles.  A warp's store or load of one
// quantity is one contiguous 256-byte segment, and the F + 1 quantities of a
// column and level lie at fixed offsets (32 q) from one address:
//   entry (k, q, col) at k LS + (col / 32) (F + 1) 32 + 32 q + col % 32,
//   LS = ceil(plane / 32) (F + 1) 32 doubles.
__host__ __device__ __forceinline__ long long fscratch_level(long long plane, int nq) {
    return (plane + 31) / 32 * nq * 32;
}
__host__ __device__ __forceinline__ long long fscratch_col(long long col, int nq) {
    return (col >> 5) * nq * 32 + (col & 31);
}
template <typename T>
cudaError_t launch_column_up(const ColumnParams<T> &p, int nf, int grid, cudaStream_t s);

cudaError_t launch_budget_reduce(const double *partials, int nblocks, int nq, int nf,
                                 double dxdy, double *out, int *status, cudaStream_t s);

cudaError_t launch_numerics(const float *in_f, const double *in_d, int n, double *widen, float *narrow,
                            double *rcp, cudaStream_t s);

template <typename T>
cudaError_t launch_stencil7(const T *in, T *out, int nx, int ny, int nz, int layout, T c, cudaStream_t s);

constexpr int COL_TPB = 128;

}  // namespace asuca
