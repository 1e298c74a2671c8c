// HEVI acoustic short steps (Sec. 1.1: sound and gravity waves in a
// second-order Runge-Kutta scheme, horizontally explicit, vertically
// implicit) of the linear acoustic-gravity system about a resting,
// horizontally uniform base state rho0(z):
//   dU/dt = -c^2 rho0 ds/dx,  dV/dt = -c^2 rho0 ds/dy,  dW/dt = -c^2 rho0f ds/dz,
//   rho0 ds/dt = -(dU/dx + dV/dy + dW/dz),          s = rho'/rho0,
// on the C grid (U at i+1/2, V at j+1/2, W at k-1/2 with rigid lids, s at the
// centres).  A short step of length h is two stages from the same start:
//   stage 1 (tau = h/2): U* = U - tau G(s),  (W*, s*) implicit with Dh(U*, V*);
//   stage 2 (tau = h):   U+ = U - tau G(s*), (W+, s+) implicit with Dh(U*, V*);
// the implicit part weights the new and old vertical terms by beta and
// 1 - beta.  Eliminating s' leaves a tridiagonal system in W' per column,
//   W'_f (1 + A_f (B_f + B_{f-1})) - A_f B_f W'_{f+1} - A_f B_{f-1} W'_{f-1}
//       = q_f - A_f (r_f - r_{f-1}),
//   s'_k = r_k - B_k (W'_{k+1} - W'_k),
// with the explicit parts r_k = s_k - (tau / rho0_k)(Dh_k + (1 - beta)(W_{k+1} - W_k)/dz_k)
// and q_f = W_f - (1 - beta) G_f (s_f - s_{f-1}).  Its matrix is the same in
// every column, so the host factorises it once per stage and a column costs
// one FMA and one multiply per face on the way up and one FMA on the way down.
//
// Mapping: one thread per (i, j) column (32 x 8 blocks), marching up (the
// horizontal terms, the explicit parts and the forward elimination, whose
// values wait in the output arrays) and back down (back substitution and s').
// In stage 1 the up pass's inputs arrive through a per-thread cp.async ring
// in shared memory, requested two levels ahead; stage 2 prefetches one level
// into registers.  The values that wait for the way down are stored with an
// L2 evict-last policy and read back with evict-first (createpolicy and
// L2::cache_hint), so they stay in L2 between the two passes instead of
// making a round trip to HBM while the streamed inputs pass through.
// The thread recomputes the neighbouring face's stage-1 momentum it needs for
// the divergence (the same operations as the neighbour's own), so a stage is
// one launch with no grid-wide dependency.  Stage 2 updates the caller's
// fields in place: every thread reads and writes only its own faces and
// column there, and reads neighbours only from the stage-1 values.
// The FP32 path computes in float throughout (the factorisation is computed
// in double on the host and rounded).
// Nested in the RK3 long step, stage 2 may write the new state to other
// arrays than its start state and adds the mass fluxes its density equation
// applies, (U*, V*, (1 - beta) W + beta W'), to the stage's mean-flux
// accumulators; the advection of the scalars then uses those means.
#include "acoustic.cuh"
#include "smem_attr.cuh"

#ifndef ACOUSTIC_RING
#define ACOUSTIC_RING 3   // levels in the shared-memory ring (2 requested ahead)
#endif

namespace asuca {

template <int N>
__device__ __forceinline__ void ac_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void ac_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <typename T>
__device__ __forceinline__ void ac_cp_async(T *dst, const T *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(sizeof(T)) : "memory");
}

// stores and loads with an L2 cache policy made by createpolicy
__device__ __forceinline__ void st_keep(float *a, float v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(double *a, double v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(a), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ float ld_last(const float *a, uint64_t pol) {
    float v;
    asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol) : "memory");
    return v;
}
__device__ __forceinline__ double ld_last(const double *a, uint64_t pol) {
    double v;
    asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol) : "memory");
    return v;
}

template <typename T, int STAGE, int D>
__global__ void __launch_bounds__(256) acoustic_kernel(const __grid_constant__ AcousticParams<T> p) {
    uint64_t pol_keep, pol_drop;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol_keep));
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol_drop));
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    if (i >= p.nx || j >= p.ny) return;
    const int nx = p.nx, nz = p.nz;
    const unsigned plane = p.plane;
    const unsigned own = (unsigned)(j * nx + i);
    const unsigned ow = (unsigned)(j * nx + (i > 0 ? i - 1 : nx - 1));
    const unsigned oe = (unsigned)(j * nx + (i < nx - 1 ? i + 1 : 0));
    const unsigned os = (unsigned)((j > 0 ? j - 1 : p.ny - 1) * nx + i);
    const unsigned on = (unsigned)((j < p.ny - 1 ? j + 1 : 0) * nx + i);
    const T *se = STAGE == 1 ? p.S : p.Ss;     // the s that drives the horizontal momenta
    T *Wo = STAGE == 1 ? p.Ws : p.Wo;
    T *So = STAGE == 1 ? p.Ss : p.So;
    const bool acc = STAGE == 2 && p.Mu != nullptr;

    // ---- up: horizontal momenta, explicit parts, forward elimination.  The
    // inputs of each level stream through a ring of D shared-memory slots
    // filled by per-thread cp.async copies, requested D - 1 levels ahead
    // (every thread copies and reads only its own slots, so no barrier is
    // needed; no store of this thread or of another one touches what a
    // request loads).  The ring keeps several levels' loads in flight without
    // holding them in registers.
    extern __shared__ __align__(16) unsigned char ac_smem[];
    T *ring = reinterpret_cast<T *>(ac_smem);
    const int tid = threadIdx.y * 32 + threadIdx.x;
    constexpr int NV = 11;   // values per level: s, W_{k+2}, s at e, n, own (stage 2), w, s; U, U_w, V, V_s
    constexpr int DR = D > 0 ? D : 1;
    auto sl = [&](int k, int v) -> T * { return ring + ((k % DR) * NV + v) * 256 + tid; };
    auto request = [&](int k) {
        if (k < nz) {
            const unsigned b = (unsigned)k * plane;
            ac_cp_async(sl(k, 0), p.S + b + own);
            if (k + 2 < nz) ac_cp_async(sl(k, 1), p.W + b + 2 * plane + own);
            else *sl(k, 1) = T(0);             // W_{k+2} at or above the lid
            ac_cp_async(sl(k, 2), se + b + oe);
            ac_cp_async(sl(k, 3), se + b + on);
            ac_cp_async(sl(k, 7), p.U + b + own);
            ac_cp_async(sl(k, 9), p.V + b + own);
            if (STAGE == 1) {
                ac_cp_async(sl(k, 5), se + b + ow);
                ac_cp_async(sl(k, 6), se + b + os);
                ac_cp_async(sl(k, 8), p.U + b + ow);
                ac_cp_async(sl(k, 10), p.V + b + os);
            } else {
                ac_cp_async(sl(k, 4), se + b + own);
                ac_cp_async(sl(k, 5), p.Us + b + own);   // stage 2: the stage-1 momenta on both faces
                ac_cp_async(sl(k, 8), p.Us + b + ow);
                ac_cp_async(sl(k, 6), p.Vs + b + own);
                ac_cp_async(sl(k, 10), p.Vs + b + os);
            }
        }
        ac_cp_commit();
    };
    struct Level { T sk, w2, c, e, w, n, s, u, uw, v, vs; };
    // without a ring (D = 0): the next level's values are loaded into registers
    auto load = [&](int k) {
        Level L;
        const unsigned b = (unsigned)k * plane;
        L.sk = p.S[b + own];
        L.w2 = (k + 2 < nz) ? p.W[b + 2 * plane + own] : T(0);
        L.e = se[b + oe];
        L.n = se[b + on];
        L.u = p.U[b + own];
        L.v = p.V[b + own];
        if (STAGE == 1) {
            L.c = L.sk;
            L.w = se[b + ow];
            L.s = se[b + os];
            L.uw = p.U[b + ow];
            L.vs = p.V[b + os];
        } else {
            L.c = se[b + own];
            L.w = p.Us[b + own];
            L.uw = p.Us[b + ow];
            L.s = p.Vs[b + own];
            L.vs = p.Vs[b + os];
        }
        return L;
    };
    auto read = [&](int k) {
        Level L;
        L.sk = *sl(k, 0);
        L.w2 = *sl(k, 1);
        L.e = *sl(k, 2);
        L.n = *sl(k, 3);
        L.c = STAGE == 1 ? L.sk : *sl(k, 4);
        L.w = *sl(k, 5);
        L.s = *sl(k, 6);
        L.u = *sl(k, 7);
        L.uw = *sl(k, 8);
        L.v = *sl(k, 9);
        L.vs = *sl(k, 10);
        return L;
    };
    Level ahead;
    if constexpr (D > 0) {
#pragma unroll 1
        for (int k = 0; k < D - 1; k++) request(k);
    } else {
        ahead = load(0);
    }
    T Wk = T(0);                               // W_k of the start state (W_0: the lid)
    T s_prev = T(0), r_prev = T(0), d_prev = T(0);
    T Wk1 = nz > 1 ? p.W[plane + own] : T(0);
#pragma unroll 1
    for (int k = 0; k < nz; k++) {
        const unsigned b = (unsigned)k * plane;
        Level cur;
        if constexpr (D > 0) {
            request(k + D - 1);                // into the slot level k-1 used
            ac_cp_wait<D - 1>();               // level k has landed
            cur = read(k);
        } else {
            cur = ahead;
            if (k + 1 < nz) ahead = load(k + 1);
        }
        const T sk = cur.sk;
        T Dh;
        if (STAGE == 1) {
            const T ue = cur.u - p.gx[k] * (cur.e - sk);
            const T uw = cur.uw - p.gx[k] * (sk - cur.w);
            const T vn = cur.v - p.gy[k] * (cur.n - sk);
            const T vs = cur.vs - p.gy[k] * (sk - cur.s);
            p.Us[b + own] = ue;
            p.Vs[b + own] = vn;
            Dh = (ue - uw) * p.rdx + (vn - vs) * p.rdy;
        } else {
            p.Uo[b + own] = cur.u - p.gx[k] * (cur.e - cur.c);
            p.Vo[b + own] = cur.v - p.gy[k] * (cur.n - cur.c);
            Dh = (cur.w - cur.uw) * p.rdx + (cur.s - cur.vs) * p.rdy;
            if (acc) {   // U*, V* of the cell's own faces
                p.Mu[b + own] = (p.acc_init ? T(0) : p.Mu[b + own]) + p.wacc * cur.w;
                p.Mv[b + own] = (p.acc_init ? T(0) : p.Mv[b + own]) + p.wacc * cur.s;
                if (k >= 1) p.Mw[b + own] = (p.acc_init ? T(0) : p.Mw[b + own]) + p.wlo * Wk;   // old W of face k
            }
        }
        const T r = sk - p.cr[k] * (Dh + p.cw[k] * (Wk1 - Wk));
        if (k >= 1) {
            const T q = Wk - p.cq[k] * (sk - s_prev);
            const T rhs = q - p.A[k] * (r - r_prev);
            const T d = (k == 1 ? rhs : rhs - p.lo[k] * d_prev) * p.inv[k];
            st_keep(Wo + b + own, d, pol_keep);   // face k waits here for the way down
            d_prev = d;
        }
        st_keep(So + b + own, r, pol_keep);
        r_prev = r;
        s_prev = sk;
        Wk = Wk1;
        Wk1 = cur.w2;
    }
    // ---- down: back substitution and s' (the values of level k-1 loaded
    // while level k is finished)
    T Wup = T(0);                              // W'_{k+1} (the lid at nz)
    T dk = nz > 1 ? ld_last(Wo + (unsigned)(nz - 1) * plane + own, pol_drop) : T(0);
    T rk = ld_last(So + (unsigned)(nz - 1) * plane + own, pol_drop);
#pragma unroll 1
    for (int k = nz - 1; k >= 0; k--) {
        const unsigned b = (unsigned)k * plane;
        T dn = T(0), rn = T(0);
        if (k >= 1) {
            rn = ld_last(So + b - plane + own, pol_drop);
            if (k >= 2) dn = ld_last(Wo + b - plane + own, pol_drop);
        }
        T Wn = T(0);
        if (k >= 1) {
            Wn = (k == nz - 1) ? dk : dk - p.cp[k] * Wup;
            if (STAGE == 2) Wo[b + own] = Wn;  // stage 2 only: nothing reads W*
            if (acc) p.Mw[b + own] += p.whi * Wn;   // new W of face k
        }
        So[b + own] = rk - p.B[k] * (Wup - Wn);
        Wup = Wn;
        dk = dn;
        rk = rn;
    }
}

template <typename T>
cudaError_t launch_acoustic_stage(const AcousticParams<T> &p, int stage, cudaStream_t s) {
    // stage 1 streams its inputs through the shared-memory ring; stage 2, whose
    // neighbour reads hit the stage-1 values in L1, keeps L1 whole and
    // prefetches one level into registers (measured faster each way)
    constexpr int D = ACOUSTIC_RING;
    constexpr size_t smem = (size_t)D * 11 * 256 * sizeof(T);
    dim3 block(32, 8), grid((p.nx + 31) / 32, (p.ny + 7) / 8);
    if (stage == 1) {
        if (smem > 48 * 1024) {
            static std::atomic<unsigned long long> attr_done{0};   // devices whose attribute is set
            const cudaError_t e = set_smem_once(acoustic_kernel<T, 1, D>, (int)smem, attr_done);
            if (e != cudaSuccess) return e;
        }
        acoustic_kernel<T, 1, D><<<grid, block, smem, s>>>(p);
    } else {
        acoustic_kernel<T, 2, 0><<<grid, block, 0, s>>>(p);
    }
    return cudaGetLastError();
}

template <typename T>
struct HeviInit {
    const T *rho;
    T *S;
    int nx, ny;
    T rho0c[MAXNZ];
};

template <typename T>
__global__ void hevi_init_kernel(const __grid_constant__ HeviInit<T> p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.nx) return;
    const size_t o = ((size_t)blockIdx.z * p.ny + blockIdx.y) * p.nx + i;
    p.S[o] = p.rho[o] / p.rho0c[blockIdx.z] - T(1);
}

template <typename T>
cudaError_t launch_hevi_init(const T *rho, const double *rho0c, T *S, int nx, int ny, int nz, cudaStream_t s) {
    HeviInit<T> p;
    p.rho = rho;
    p.S = S;
    p.nx = nx;
    p.ny = ny;
    for (int k = 0; k < MAXNZ; k++) p.rho0c[k] = k < nz ? (T)rho0c[k] : T(1);
    dim3 grid((nx + 127) / 128, ny, nz);
    hevi_init_kernel<T><<<grid, 128, 0, s>>>(p);
    return cudaGetLastError();
}

template cudaError_t launch_hevi_init<float>(const float *, const double *, float *, int, int, int, cudaStream_t);
template cudaError_t launch_hevi_init<double>(const double *, const double *, double *, int, int, int, cudaStream_t);
template cudaError_t launch_acoustic_stage<float>(const AcousticParams<float> &, int, cudaStream_t);
template cudaError_t launch_acoustic_stage<double>(const AcousticParams<double> &, int, cudaStream_t);

}  // namespace asuca
