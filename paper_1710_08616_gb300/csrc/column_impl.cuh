// Column physics (per-column device code), one thread per (i, j) column (the coarse per-column
// granularity of Sec. 1.2 "Parallelization Granularity", Fig. 1 and 2), and
// the FP64 budget sums.
//
// Per column, after the three RK stages (Lie splitting, once per long step):
//   top-down pass, k = nz-1 .. 0:
//     (i)   implicit theta relaxation   theta <- (theta + r theta_ref) / (1 + r)
//     (ii)  implicit sedimentation      (rho q)_k <- ((rho q)_k dz_k + dt P_{k+1/2}) / (dz_k + dt v),
//                                       P_{k-1/2} = v (rho q)_k; P_{-1/2} rains out
//     (iii) forward elimination of the implicit vertical diffusion
//           A phi = d, a_k = -g_{k-1/2}, c_k = -g_{k+1/2},
//           b_k = rho_k dz_k + g_{k-1/2} + g_{k+1/2}, d_k = dz_k (rho phi)_k,
//           run from the top down (the mirror of the textbook Thomas order),
//           one factorisation shared by rho*theta and every tracer
//   bottom-up pass: back substitution, (rho phi)_k = rho_k phi_k.
// The elimination works on scaled unknowns so that each field costs one
// FMA per level on the way down and one FMA plus one multiply on the way up:
//   e_k = x_k + alpha_k e_{k+1},  alpha_k = g_{k+1/2} m_{k+1} dz_{k+1} / dz_k
//   z_k = e_k + gamma_k z_{k-1},  gamma_k = g_{k-1/2} m_{k-1} dz_{k-1} / dz_k
//   (rho phi)_k = sigma_k z_k,    sigma_k = rho_k dz_k m_k,   m_k = 1 / pivot_k
// Per field and level that is two FP64 operations; the shared factorisation
// costs about twelve (its reciprocal three of them).  Float inputs are widened and the result narrowed on
// the integer pipe (the hardware conversions issue on the slow FP64 pipe);
// for float fields the final multiply by sigma_k is done in float.
// (x_k is the incoming rho*phi; d''_k = dz_k m_k e_k and phi_k = dz_k m_k z_k
// are the usual eliminated right-hand side and solution).  The whole solve
// runs in double in both precisions; a float result is rounded once.
//
// The per-level e_k, m_k, gamma_k live in a scratch area indexed by the
// thread's slot.  The grid is persistent (one resident wave, a grid-stride
// loop over columns), so the scratch is as large as the columns in flight
// and stays resident in L2 while each slot reuses it column after column.
#pragma once

#include "common.cuh"

namespace asuca {

// Budget partial of one column: sum_k f_k dz_k.  In double for the FP64 path;
// for float fields the per-column sum is carried as a compensated float pair
// (TwoProduct by FMA for f * dz_hi, Neumaier's compensated summation) and
// widened once per column, which keeps double-precision accuracy without a
// conversion and an FP64 operation per cell.
template <typename T> struct ColSum;
template <> struct ColSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double f, double dz, float, float) { s = fma(f, dz, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct ColSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float f, double, float dz_hi, float dz_lo) {
        const float p = f * dz_hi;
        const float pe = fmaf(f, dz_hi, -p);          // exact error of the product
        c = fmaf(f, dz_lo, c + pe);                   // small terms go to the compensation
        const float t = s + p;
        c += (fabsf(s) >= fabsf(p)) ? ((s - t) + p) : ((p - t) + s);
        s = t;
    }
    __device__ __forceinline__ double value() const { return f2d_bits(s) + f2d_bits(c); }
};

template <typename T> __device__ __forceinline__ T scale_out(double z, double sigma, float sigma_f);
// FP64 path: the rescaled unknown times sigma in double.
template <> __device__ __forceinline__ double scale_out<double>(double z, double sigma, float) { return sigma * z; }
// FP32 path: z rounded once to float (integer-pipe rounding), times sigma in float.
template <> __device__ __forceinline__ float scale_out<float>(double z, double, float sigma_f) {
    return d2f_bits(z) * sigma_f;
}

// The column pass of one column (col = j * nx + i); sc points at the
// thread's scratch slot (stride nslots between entries).  cs receives the
// column's budget partials when p.budgets is set.
template <typename T, int NF>
__device__ __forceinline__ void column_one(const ColumnParams<T> &p, long long col, double *sc, long long nslots,
                                           ColSum<T> (&cs)[NF]) {
    constexpr int NT = NF - 1;
    constexpr int NQ = NF + 1;                    // m, gamma, e[NT]
    const int nz = p.nz;
    const long long plane = p.plane;
    // indices checked in the bounds-check build: fields [nz][plane], the
    // thread's scratch slot (its entries nslots apart, nz NQ of them), the
    // adjoint's record [nz][F + 2][plane], the precipitation [plane]
    auto yi = [&](long long i) -> long long {
        ASUCA_BC(i, (long long)nz * plane, p.status);
        return i;
    };
    auto si = [&](long long i) -> long long {
#ifdef ASUCA_BOUNDS_CHECK
        long long t = (long long)(sc - p.scratch) + i;
        ASUCA_BC(t, (long long)nz * NQ * nslots, p.status);
        i = t - (long long)(sc - p.scratch);
#endif
        return i;
    };
    auto ri = [&](long long i) -> long long {
        ASUCA_BC(i, (long long)nz * (NF + 2) * plane, p.status);
        return i;
    };
    long long pc = col;
    ASUCA_BC(pc, plane, p.status);
    if (p.do_phys) {
        double g_hi = 0.0, m_up = 0.0;
        double e_up[NT];
#pragma unroll
        for (int f = 0; f < NT; f++) e_up[f] = 0.0;
        T P = T(0);
        long long o = (long long)(nz - 1) * plane + col;
        T rho = p.y[0][yi(o)];
        T rho_dn = (nz > 1) ? p.y[0][yi(o - plane)] : T(0);
        double rd = to_f64(rho);
        T x[NT];
#pragma unroll
        for (int f = 0; f < NT; f++) x[f] = p.y[f + 1][yi(o)];
        for (int k = nz - 1; k >= 0; k--, o -= plane) {
            // prefetch the level below (and rho two below) while this level computes
            T xn[NT];
            T rho_dn2 = T(0);
            if (k > 0) {
#pragma unroll
                for (int f = 0; f < NT; f++) xn[f] = p.y[f + 1][yi(o - plane)];
                if (k > 1) rho_dn2 = p.y[0][yi(o - 2 * plane)];
            }
            // (i) relaxation of theta
            if (p.do_relax) {
                T th = x[0] / rho;
                th = (th + p.relax_r * p.thref[k]) * p.relax_inv;
                x[0] = rho * th;
            }
            // (ii) sedimentation of one tracer, top-down
            if (p.do_sed) {
#pragma unroll
                for (int f = 1; f < NT; f++) {
                    if (f + 1 == p.sed) {
                        x[f] = (x[f] * p.dzT[k] + p.sed_dt * P) * p.sedr[k];
                        P = p.sed_v * x[f];
                    }
                }
                if (k == 0) p.precip_col[pc] += p.dt * to_f64(P) * p.dxdy;
            }
            if (p.budgets) cs[0].add(rho, p.dz[k], p.dzT[k], p.dzlo[k]);
            const double rd_dn = (k > 0) ? to_f64(rho_dn) : 0.0;
            if (p.do_diff) {
                // (iii) forward elimination, top-down, on scaled unknowns
                const double g_lo = (k > 0) ? p.kc[k - 1] * (rd_dn + rd) : 0.0;
                const double b = fma(rd, p.dz[k], g_lo + g_hi);
                const double t = g_hi * m_up;
                const double m = rcp_f64(fma(-g_hi, t, b));
                const double alpha = t * p.dzr_up[k];
                sc[si((long long)(k * NQ + 0) * nslots)] = m;
                const double gam = (k < nz - 1) ? g_hi * m * p.dzr_dn[k + 1] : 0.0;
                if (k < nz - 1) sc[si((long long)((k + 1) * NQ + 1) * nslots)] = gam;
                if (p.rec) {   // the adjoint's record of the factorisation
                    p.rec[ri((long long)(k * (NF + 2) + 0) * plane + col)] = m;
                    p.rec[ri((long long)(k * (NF + 2) + 1) * plane + col)] = alpha;
                    if (k < nz - 1) p.rec[ri((long long)((k + 1) * (NF + 2) + 2) * plane + col)] = gam;
                }
#pragma unroll
                for (int f = 0; f < NT; f++) {
                    const double e = fma(alpha, e_up[f], to_f64(x[f]));
                    sc[si((long long)(k * NQ + 2 + f) * nslots)] = e;
                    e_up[f] = e;
                }
                g_hi = g_lo;
                m_up = m;
            } else {
                if (p.do_relax) p.y[1][yi(o)] = x[0];
                if (p.do_sed) {
#pragma unroll
                    for (int f = 1; f < NT; f++)
                        if (f + 1 == p.sed) p.y[f + 1][yi(o)] = x[f];
                }
                if (p.budgets) {
#pragma unroll
                    for (int f = 0; f < NT; f++) cs[f + 1].add(x[f], p.dz[k], p.dzT[k], p.dzlo[k]);
                }
            }
            if (k > 0) {
#pragma unroll
                for (int f = 0; f < NT; f++) x[f] = xn[f];
            }
            rho = rho_dn;
            rho_dn = rho_dn2;
            rd = rd_dn;
        }
        if (p.do_diff) {
            // back substitution, bottom-up; sigma_k = rho_k dz_k m_k
            double z[NT];
#pragma unroll
            for (int f = 0; f < NT; f++) z[f] = 0.0;
            long long ob = col;
            double mk = sc[si(0)], gk = 0.0;
            double ek[NT];
#pragma unroll
            for (int f = 0; f < NT; f++) ek[f] = sc[si((long long)(2 + f) * nslots)];
            T rk = p.y[0][yi(ob)];
            for (int k = 0; k < nz; k++, ob += plane) {
                double mn = 0.0, gn = 0.0, en[NT];
                T rn = T(0);
                if (k + 1 < nz) {   // prefetch level k+1
                    mn = sc[si((long long)((k + 1) * NQ + 0) * nslots)];
                    gn = sc[si((long long)((k + 1) * NQ + 1) * nslots)];
#pragma unroll
                    for (int f = 0; f < NT; f++) en[f] = sc[si((long long)((k + 1) * NQ + 2 + f) * nslots)];
                    rn = p.y[0][yi(ob + plane)];
                }
                const double sigma = to_f64(rk) * p.dz[k] * mk;
                // float path: sigma in float from rho (float), dz and m rounded once
                const float sf = (sizeof(T) == 4) ? (float)rk * (float)p.dzT[k] * d2f_bits(mk) : 0.f;
#pragma unroll
                for (int f = 0; f < NT; f++) {
                    z[f] = fma(gk, z[f], ek[f]);
                    if (p.rec) p.rec[ri((size_t)(k * (NF + 2) + 3 + f) * plane + col)] = z[f];
                    const T u = scale_out<T>(z[f], sigma, sf);
                    p.y[f + 1][yi(ob)] = u;
                    if (p.budgets) cs[f + 1].add(u, p.dz[k], p.dzT[k], p.dzlo[k]);
                }
                if (k + 1 < nz) {
                    mk = mn;
                    gk = gn;
#pragma unroll
                    for (int f = 0; f < NT; f++) ek[f] = en[f];
                    rk = rn;
                }
            }
        }
    } else if (p.budgets) {
        for (int k = 0; k < nz; k++) {
            const long long o = (long long)k * plane + col;
#pragma unroll
            for (int f = 0; f < NF; f++) cs[f].add(p.y[f][yi(o)], p.dz[k], p.dzT[k], p.dzlo[k]);
        }
    }
}

}  // namespace asuca

namespace asuca {

// The per-level constants of the top-down column pass, gathered into one
// record per level (ColDownHook reads a level's record from shared memory in
// three 16-byte loads instead of one constant-bank load per value).
template <typename T>
struct __align__(16) ColLevel {
    double kc_lo;     // kc[k - 1]: dt K / dzc / 2 of face k - 1/2 (0 at k = 0)
    double dz;        // dz_k
    double dzr_up;    // dz_{k+1} / dz_k
    double dzr_dn1;   // dzr_dn[k + 1] = dz_k / dz_{k+1} (0 at the top level)
    T thref, dzT, sedr, pad;   // theta_ref(z_k), dz_k and 1 / (dz_k + dt v) in T
};

// Fill the records of levels 0 .. nz-1 (threads tid of nthr share the work).
template <typename T>
__device__ __forceinline__ void fill_col_levels(const ColumnParams<T> &c, ColLevel<T> *tab, int tid, int nthr) {
    for (int k = tid; k < c.nz; k += nthr) {
        ColLevel<T> L;
        L.kc_lo = k > 0 ? c.kc[k - 1] : 0.0;
        L.dz = c.dz[k];
        L.dzr_up = c.dzr_up[k];
        L.dzr_dn1 = k + 1 < c.nz ? c.dzr_dn[k + 1] : 0.0;
        L.thref = c.thref[k];
        L.dzT = c.dzT[k];
        L.sedr = c.sedr[k];
        L.pad = T(0);
        tab[k] = L;
    }
}

// ------------------------------------------------------------------ column pass fused into the stages

// The top-down half of the column pass runs inside the stage kernels, which
// march the levels from the top down and hand each level's result to a hook:
// hook.level(k, out, valid, rho_next, rho_h), where out is the stage's result,
// rho_next the density result of the next level of the march, and rho_h the
// density after the whole step when the hook asks for it (own_rho).  Hooks
// with keep_output let the stage write its result as usual.
//
// The per-level values m, gamma, e_f go to the fused scratch (fscratch_level /
// fscratch_col: quantity q = 0 m, 1 gamma, 2 + f e_f) for column_up_kernel's
// bottom-up back substitution.  Two arrangements, with the same operations
// as column_one's top-down pass and so the same results:
//  * ColDownHook in stage 3: relaxation, sedimentation, factorisation and
//    elimination of every level;
//  * FactorHook in stage 2 and SweepHook in stage 3: the factorisation depends
//    only on the density after the step, which the mass fluxes fix before the
//    step begins (the density's flux is M), so stage 2 computes it (m, gamma
//    to the scratch, alpha to an array of its own) and stage 3 keeps only the
//    relaxation, the sedimentation and the nine-field elimination sweep.  The
//    FP64 work is then split between two kernels whose FP32 stencils it
//    overlaps.
// tab holds the per-level records (ColLevel) in shared memory.

// Relaxation and sedimentation of one level (top-down), in T.
template <typename T, int NF>
__device__ __forceinline__ void column_physics_level(const ColumnParams<T> &c, const ColLevel<T> &L, int k, T rho,
                                                     T (&x)[NF - 1], T &P, unsigned own) {
    constexpr int NT = NF - 1;
    // (i) relaxation of theta
    if (c.do_relax) {
        T th = x[0] / rho;
        th = (th + c.relax_r * L.thref) * c.relax_inv;
        x[0] = rho * th;
    }
    // (ii) sedimentation of one tracer, top-down (the last tracer as a
    // compile-time index, any other by compare)
    if (c.do_sed) {
        if (c.sed == NF - 1) {
            x[NT - 1] = (x[NT - 1] * L.dzT + c.sed_dt * P) * L.sedr;
            P = c.sed_v * x[NT - 1];
        } else {
#pragma unroll
            for (int f = 1; f < NT; f++) {
                if (f + 1 == c.sed) {
                    x[f] = (x[f] * L.dzT + c.sed_dt * P) * L.sedr;
                    P = c.sed_v * x[f];
                }
            }
        }
        if (k == 0) {
            unsigned o = own;
            ASUCA_BC(o, c.plane, c.status);
            c.precip_col[o] += c.dt * to_f64(P) * c.dxdy;
        }
    }
}

// The scratch entries of level k of the column whose entries start at sc
// (a pointer into c.scratch): the checked build tests that quantities 0 ..
// hi_q of the level lie inside the fused scratch.
template <typename T>
__device__ __forceinline__ double *fscratch_at(const ColumnParams<T> &c, double *sc, int k, size_t ls, int hi_q) {
#ifdef ASUCA_BOUNDS_CHECK
    long long ai = (long long)(sc - c.scratch) + (long long)k * (long long)ls;
    ASUCA_BC(ai, (long long)c.nz * (long long)ls - 32LL * hi_q, c.status);
    return c.scratch + ai;
#else
    (void)c;
    (void)hi_q;
    return sc + (size_t)k * ls;
#endif
}

// The factorisation of one level (top-down, scaled unknowns): stores m and
// the next level's gamma at a (the level's scratch entries, ls the level
// stride), carries g and m to the next level, returns alpha.
template <typename T>
__device__ __forceinline__ double factor_level(const ColLevel<T> &L, int k, int nz, T rho, T rho_next, double &g_hi,
                                               double &m_up, double *a, size_t ls, const double *bc_base = nullptr,
                                               long long bc_extent = 0, int *bc_status = nullptr) {
    (void)bc_base;
    (void)bc_extent;
    (void)bc_status;
    const double rd = to_f64(rho);
    const double rd_dn = (k > 0) ? to_f64(rho_next) : 0.0;
    const double g_lo = (k > 0) ? L.kc_lo * (rd_dn + rd) : 0.0;
    const double b = fma(rd, L.dz, g_lo + g_hi);
    const double t = g_hi * m_up;
    const double m = rcp_f64(fma(-g_hi, t, b));
    const double alpha = t * L.dzr_up;
    a[0] = m;
    if (k < nz - 1) {
        size_t gi = ls + 32;   // gamma of level k + 1
#ifdef ASUCA_BOUNDS_CHECK
        // a + gi inside [base, base + extent)
        long long ga = (long long)(a - bc_base) + (long long)gi;
        ASUCA_BC(ga, bc_extent, bc_status);
        gi = (size_t)(ga - (long long)(a - bc_base));
#endif
        a[gi] = g_hi * m * L.dzr_dn1;
    }
    g_hi = g_lo;
    m_up = m;
    return alpha;
}

// Relaxation, sedimentation, factorisation and elimination in stage 3.  The
// density result is written to the state here; rho*theta and the tracers are
// written by the back substitution.
template <typename T, int NF>
struct ColDownHook {
    static constexpr bool active = true, keep_output = false, own_rho = false, defers = false;
    static constexpr int NT = NF - 1;
    static constexpr int NQ = NF + 1;   // m, gamma, e[NT]
    const ColumnParams<T> &c;
    const ColLevel<T> *tab;
    T *rho_out;
    double *sc;
    size_t pl, ls;
    unsigned own;
    double g_hi, m_up;
    double e_up[NT];
    T P;

    __device__ __forceinline__ ColDownHook(const ColumnParams<T> &cp, const ColLevel<T> *tab_, T *rho, unsigned own_)
        : c(cp), tab(tab_), rho_out(rho), sc(cp.scratch + fscratch_col(own_, NQ)), pl((size_t)cp.plane),
          ls((size_t)fscratch_level(cp.plane, NQ)), own(own_), g_hi(0.0), m_up(0.0), P(T(0)) {
#pragma unroll
        for (int f = 0; f < NT; f++) e_up[f] = 0.0;
    }

    template <typename U, int NF2>
    __device__ __forceinline__ void level(int k, const U (&out)[NF2], bool valid, U rho_next, U) {
        static_assert(NF2 == NF, "field count");
        if (!valid) return;
        const T rho = out[0];
        size_t ro = (size_t)k * pl + own;
        ASUCA_BC(ro, (long long)c.nz * (long long)pl, c.status);
        rho_out[ro] = rho;
        const ColLevel<T> L = tab[k];
        T x[NT];
#pragma unroll
        for (int f = 0; f < NT; f++) x[f] = out[f + 1];
        column_physics_level<T, NF>(c, L, k, rho, x, P, own);
        // (iii) forward elimination on scaled unknowns
        double *a = fscratch_at(c, sc, k, ls, NQ - 1);
        const double alpha = factor_level<T>(L, k, c.nz, rho, rho_next, g_hi, m_up, a, ls, c.scratch,
                                             (long long)c.nz * (long long)ls, c.status);
#pragma unroll
        for (int f = 0; f < NT; f++) {
            const double e = fma(alpha, e_up[f], to_f64(x[f]));
            a[32 * (2 + f)] = e;
            e_up[f] = e;
        }
    }
    __device__ __forceinline__ void early() {}
    __device__ __forceinline__ void done(bool) {}
};

// The factorisation in stage 2 (the stage's own result is written as usual):
// from the density after the step (rho_h, rho_next), m and gamma to the fused
// scratch and alpha to c.alpha ([nz][plane]).  With LAG a level's
// factorisation waits for the next level's early() and so runs beside that
// level's faces (its dependent FP64 chain then interleaves with independent
// stencil work); the last level's runs in done().
template <typename T, int NF, bool LAG = false>
struct FactorHook {
    static constexpr bool active = true, keep_output = true, own_rho = true, defers = LAG;
    static constexpr int NQ = NF + 1;
    const ColumnParams<T> &c;
    const ColLevel<T> *tab;
    double *sc, *alpha_out;
    size_t pl, ls;
    double g_hi, m_up;

    __device__ __forceinline__ FactorHook(const ColumnParams<T> &cp, const ColLevel<T> *tab_, unsigned own)
        : c(cp), tab(tab_), sc(cp.scratch + fscratch_col(own, NQ)), alpha_out(cp.alpha + own),
          pl((size_t)cp.plane), ls((size_t)fscratch_level(cp.plane, NQ)), g_hi(0.0), m_up(0.0) {}

    struct Pending {   // LAG: the level whose factorisation is pending, and its densities
        int k = -1;
        T rh = T(0), rn = T(0);
    };
    struct NoPending {};
    typename std::conditional<LAG, Pending, NoPending>::type pend;

    template <typename U, int NF2>
    __device__ __forceinline__ void level(int k, const U (&)[NF2], bool valid, U rho_next, U rho_h) {
        if (!valid) return;
        if constexpr (LAG) {
            pend.k = k;
            pend.rh = rho_h;
            pend.rn = rho_next;
        } else {
            run(k, rho_h, rho_next);
        }
    }
    __device__ __forceinline__ void early() {
        if constexpr (LAG) {
            if (pend.k >= 0) {
                run(pend.k, pend.rh, pend.rn);
                pend.k = -1;
            }
        }
    }
    __device__ __forceinline__ void run(int k, T rho_h, T rho_next) {
        const ColLevel<T> L = tab[k];
        size_t ao = (size_t)k * pl;
#ifdef ASUCA_BOUNDS_CHECK
        long long aa = (long long)(alpha_out - c.alpha) + (long long)ao;
        ASUCA_BC(aa, (long long)c.nz * (long long)pl, c.status);
        ao = (size_t)(aa - (long long)(alpha_out - c.alpha));
#endif
        alpha_out[ao] = factor_level<T>(L, k, c.nz, rho_h, rho_next, g_hi, m_up, fscratch_at(c, sc, k, ls, 1), ls,
                                        c.scratch, (long long)c.nz * (long long)ls, c.status);
    }
    __device__ __forceinline__ void done(bool) { early(); }
};

// Relaxation, sedimentation and the elimination sweep in stage 3, after
// FactorHook in stage 2 (alpha read from c.alpha one level ahead).
template <typename T, int NF>
struct SweepHook {
    static constexpr bool active = true, keep_output = false, own_rho = false, defers = false;
    static constexpr int NT = NF - 1;
    static constexpr int NQ = NF + 1;
    const ColumnParams<T> &c;
    const ColLevel<T> *tab;
    T *rho_out;
    double *sc;
    const double *alpha_in;
    size_t pl, ls;
    unsigned own;
    double alpha_k;   // alpha of the level the march reaches next
    double e_up[NT];
    T P;

    __device__ __forceinline__ SweepHook(const ColumnParams<T> &cp, const ColLevel<T> *tab_, T *rho, unsigned own_)
        : c(cp), tab(tab_), rho_out(rho), sc(cp.scratch + fscratch_col(own_, NQ)), alpha_in(cp.alpha + own_),
          pl((size_t)cp.plane), ls((size_t)fscratch_level(cp.plane, NQ)), own(own_), P(T(0)) {
        alpha_k = alpha_in[alpha_index(cp.nz - 1)];
#pragma unroll
        for (int f = 0; f < NT; f++) e_up[f] = 0.0;
    }

    // offset of level k's alpha from alpha_in (checked against the [nz][plane] array)
    __device__ __forceinline__ long long alpha_index(int k) const {
        long long a = (long long)k * (long long)pl;
#ifdef ASUCA_BOUNDS_CHECK
        long long t = a + own;
        ASUCA_BC(t, (long long)c.nz * (long long)pl, c.status);
        a = t - own;
#endif
        return a;
    }

    template <typename U, int NF2>
    __device__ __forceinline__ void level(int k, const U (&out)[NF2], bool valid, U, U) {
        static_assert(NF2 == NF, "field count");
        if (!valid) return;
        const double alpha = alpha_k;
        if (k > 0) alpha_k = alpha_in[alpha_index(k - 1)];
        const T rho = out[0];
        size_t ro = (size_t)k * pl + own;
        ASUCA_BC(ro, (long long)c.nz * (long long)pl, c.status);
        rho_out[ro] = rho;
        const ColLevel<T> L = tab[k];
        T x[NT];
#pragma unroll
        for (int f = 0; f < NT; f++) x[f] = out[f + 1];
        column_physics_level<T, NF>(c, L, k, rho, x, P, own);
        double *a = fscratch_at(c, sc, k, ls, NQ - 1);
#pragma unroll
        for (int f = 0; f < NT; f++) {
            const double e = fma(alpha, e_up[f], to_f64(x[f]));
            a[32 * (2 + f)] = e;
            e_up[f] = e;
        }
    }
    __device__ __forceinline__ void early() {}
    __device__ __forceinline__ void done(bool) {}
};

// The bottom-up half of the column pass after ColDownHook, for one column:
// back substitution from the fused scratch (fscratch_level / fscratch_col),
// (rho phi)_k = sigma_k z_k for rho*theta and every tracer (column_one's
// bottom-up pass, operation for operation), and the column's budget partials
// in cs when p.budgets is set.  Float results: the level's nine solutions and
// its m are narrowed together (d2f_fast, the exact path for the whole level
// when one of them lies outside the float normal range).
template <typename T, int NF>
__device__ __forceinline__ void column_up_one(const ColumnParams<T> &p, long long col, ColSum<T> (&cs)[NF]) {
    constexpr int NT = NF - 1;
    constexpr int NQ = NF + 1;
    const size_t pl = (size_t)p.plane;
    const size_t ls = (size_t)fscratch_level(p.plane, NQ);
    const int nz = p.nz;
    double *sc = p.scratch + fscratch_col(col, NQ);
    double z[NT];
#pragma unroll
    for (int f = 0; f < NT; f++) z[f] = 0.0;
    size_t ob = (size_t)col;
    const double *a0 = fscratch_at(p, sc, 0, ls, NQ - 1);
    double mk = a0[0], gk = 0.0;
    double ek[NT];
#pragma unroll
    for (int f = 0; f < NT; f++) ek[f] = a0[32 * (2 + f)];
    size_t o0 = ob;
    ASUCA_BC(o0, (long long)nz * (long long)pl, p.status);
    T rk = p.y[0][o0];
    for (int k = 0; k < nz; k++, ob += pl) {
        double mn = 0.0, gn = 0.0, en[NT];
        T rn = T(0);
        if (k + 1 < nz) {   // prefetch level k+1
            const double *a = fscratch_at(p, sc, k + 1, ls, NQ - 1);
            mn = a[0];
            gn = a[32];
#pragma unroll
            for (int f = 0; f < NT; f++) en[f] = a[32 * (2 + f)];
            size_t on = ob + pl;
            ASUCA_BC(on, (long long)nz * (long long)pl, p.status);
            rn = p.y[0][on];
        }
        if (p.budgets) cs[0].add(rk, p.dz[k], p.dzT[k], p.dzlo[k]);
#pragma unroll
        for (int f = 0; f < NT; f++) z[f] = fma(gk, z[f], ek[f]);
        T u[NT];
        if constexpr (sizeof(T) == 4) {
            // sigma in float from rho, dz and m rounded once; z rounded once
            bool ok = true;
            float zf[NT];
            float mf = d2f_fast(mk, ok);
#pragma unroll
            for (int f = 0; f < NT; f++) zf[f] = d2f_fast(z[f], ok);
            if (!ok) {
                mf = d2f_bits(mk);
#pragma unroll
                for (int f = 0; f < NT; f++) zf[f] = d2f_bits(z[f]);
            }
            const float sf = rk * p.dzT[k] * mf;
#pragma unroll
            for (int f = 0; f < NT; f++) u[f] = zf[f] * sf;
        } else {
            const double sigma = rk * p.dz[k] * mk;
#pragma unroll
            for (int f = 0; f < NT; f++) u[f] = sigma * z[f];
        }
        size_t os = ob;
        ASUCA_BC(os, (long long)nz * (long long)pl, p.status);
#pragma unroll
        for (int f = 0; f < NT; f++) {
            p.y[f + 1][os] = u[f];
            if (p.budgets) cs[f + 1].add(u[f], p.dz[k], p.dzT[k], p.dzlo[k]);
        }
        if (k + 1 < nz) {
            mk = mn;
            gk = gn;
#pragma unroll
            for (int f = 0; f < NT; f++) ek[f] = en[f];
            rk = rn;
        }
    }
}

}  // namespace asuca
