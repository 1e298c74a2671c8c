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
// The thread recomputes the neighbouring face's stage-1 momentum it needs for
// the divergence (the same operations as the neighbour's own), so a stage is
// one launch with no grid-wide dependency.  Stage 2 updates the caller's
// fields in place: every thread reads and writes only its own faces and
// column there, and reads neighbours only from the stage-1 values.
// The FP32 path computes in float throughout (the factorisation is computed
// in double on the host and rounded).
#include "acoustic.cuh"

namespace asuca {

template <typename T, int STAGE>
__global__ void __launch_bounds__(256) acoustic_kernel(const __grid_constant__ AcousticParams<T> p) {
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
    T *Wo = STAGE == 1 ? p.Ws : p.W;
    T *So = STAGE == 1 ? p.Ss : p.S;

    // ---- up: horizontal momenta, explicit parts, forward elimination
    T Wk = T(0);                               // W_k of the start state (W_0: the lid)
    T s_prev = T(0), r_prev = T(0), d_prev = T(0);
    T Wk1 = nz > 1 ? p.W[plane + own] : T(0);
#pragma unroll 1
    for (int k = 0; k < nz; k++) {
        const unsigned b = (unsigned)k * plane;
        const T sk = p.S[b + own];
        // W_{k+2} one level ahead (the lid at nz reads as zero)
        const T Wk2 = (k + 2 < nz) ? p.W[b + 2 * plane + own] : T(0);
        T Dh;
        if (STAGE == 1) {
            const T sE = se[b + oe], sW = se[b + ow], sN = se[b + on], sS = se[b + os];
            const T ue = p.U[b + own] - p.gx[k] * (sE - sk);
            const T uw = p.U[b + ow] - p.gx[k] * (sk - sW);
            const T vn = p.V[b + own] - p.gy[k] * (sN - sk);
            const T vs = p.V[b + os] - p.gy[k] * (sk - sS);
            p.Us[b + own] = ue;
            p.Vs[b + own] = vn;
            Dh = (ue - uw) * p.rdx + (vn - vs) * p.rdy;
        } else {
            const T sc = se[b + own], sE = se[b + oe], sN = se[b + on];
            p.U[b + own] = p.U[b + own] - p.gx[k] * (sE - sc);
            p.V[b + own] = p.V[b + own] - p.gy[k] * (sN - sc);
            Dh = (p.Us[b + own] - p.Us[b + ow]) * p.rdx + (p.Vs[b + own] - p.Vs[b + os]) * p.rdy;
        }
        const T r = sk - p.cr[k] * (Dh + p.cw[k] * (Wk1 - Wk));
        if (k >= 1) {
            const T q = Wk - p.cq[k] * (sk - s_prev);
            const T rhs = q - p.A[k] * (r - r_prev);
            const T d = (k == 1 ? rhs : rhs - p.lo[k] * d_prev) * p.inv[k];
            Wo[b + own] = d;                   // face k waits here for the way down
            d_prev = d;
        }
        So[b + own] = r;
        r_prev = r;
        s_prev = sk;
        Wk = Wk1;
        Wk1 = Wk2;
    }
    // ---- down: back substitution and s'
    T Wup = T(0);                              // W'_{k+1} (the lid at nz)
#pragma unroll 1
    for (int k = nz - 1; k >= 0; k--) {
        const unsigned b = (unsigned)k * plane;
        T Wn = T(0);
        if (k >= 1) {
            const T d = Wo[b + own];
            Wn = (k == nz - 1) ? d : d - p.cp[k] * Wup;
            if (STAGE == 2) Wo[b + own] = Wn;  // stage 2 only: nothing reads W*
        }
        So[b + own] = So[b + own] - p.B[k] * (Wup - Wn);
        Wup = Wn;
    }
}

template <typename T>
cudaError_t launch_acoustic_stage(const AcousticParams<T> &p, int stage, cudaStream_t s) {
    dim3 block(32, 8), grid((p.nx + 31) / 32, (p.ny + 7) / 8);
    if (stage == 1) acoustic_kernel<T, 1><<<grid, block, 0, s>>>(p);
    else acoustic_kernel<T, 2><<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

template cudaError_t launch_acoustic_stage<float>(const AcousticParams<float> &, int, cudaStream_t);
template cudaError_t launch_acoustic_stage<double>(const AcousticParams<double> &, int, cudaStream_t);

}  // namespace asuca
