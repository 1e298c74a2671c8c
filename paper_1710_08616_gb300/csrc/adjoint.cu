// Adjoint of the step (the gradient engine of a 4D-Var-style assimilation):
// the transpose of one RK stage's right-hand side, and the transpose of the
// column pass.  Limiter branches are the ones the forward pass recorded, so
// each face is differentiated along the branch it took; with the branch fixed
// the limiter increment is linear, L = a d0 + b d1.
//
// Stage transpose, for mu = c_s * lambda_s (lambda_s the adjoint of the
// stage output) and the stage input Y with phi = rho*phi / rho:
//   face a+1/2 with flux F = M face(phi):  lambda_F = mu(a+1)/D(a+1) - mu(a)/D(a)
//   lambda_phi(c) = sum over faces whose stencil holds c of lambda_F M dface/dphi(c)
//   lambda(rho phi)(c) = lambda_phi / rho,   lambda(rho)(c) -= lambda_phi phi / rho
//   gradient of M at the face += lambda_F(rho) + sum_f lambda_F(f) face_f
// It is written as a gather: the thread of cell c visits the four faces per
// direction whose stencil can hold c, so no two threads write the same value
// and the result does not depend on scheduling.
#include "adjoint_params.cuh"

namespace asuca {

template <typename T, int NF, int LIM>
__global__ void __launch_bounds__(128) adj_stage_kernel(const __grid_constant__ AdjStageParams<T> p) {
    constexpr int NT = NF - 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    if (i >= nx || j >= ny) return;
    const long long plane = p.plane;
    int ix[5], jy[5];
#pragma unroll
    for (int q = 0; q < 5; q++) {
        ix[q] = wrap_index(i + q - 2, nx);
        jy[q] = wrap_index(j + q - 2, ny);
    }
    // planar offsets (caller layout) of the cells i-2..i+2 (row j) and j-2..j+2 (column i)
    long long ox[5], oy[5];
#pragma unroll
    for (int q = 0; q < 5; q++) {
        ox[q] = (long long)j * nx + ix[q];
        oy[q] = (long long)jy[q] * nx + i;
    }
    // the same cells in the layout of the stage input
    long long sx[5], sy[5];
#pragma unroll
    for (int q = 0; q < 5; q++) {
        sx[q] = (long long)(j + p.ys_oy) * p.ys_pitch + ix[q] + p.ys_ox;
        sy[q] = (long long)(jy[q] + p.ys_oy) * p.ys_pitch + i + p.ys_ox;
    }
    const T cs = p.cs, rdx = p.rdx, rdy = p.rdy;

    for (int k = 0; k < nz; k++) {
        const long long kb = (long long)k * plane, skb = (long long)k * p.ys_plane;
        const long long own = kb + ox[2];
        // mass fluxes of the four faces per direction that touch cell c; face a+1/2 is stored at cell a
        T mxf[4], myf[4], mzf[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            mxf[q] = p.mu[kb + ox[q]];
            myf[q] = p.mv[kb + oy[q]];
            const int a = k + q - 2;
            mzf[q] = (a >= 0 && a <= nz - 2) ? p.mw[(long long)(a + 1) * plane + ox[2]] : T(0);
        }
        const T rho = p.ys[0][skb + sx[2]];
        const T rr = recip(rho);
        T vrho = T(0);
        // --- density: no phi, only the gradient of M
        T lf0x, lf0y, lf0z;
        {
            const T m0 = p.lam[0][own], mxp = p.lam[0][kb + ox[3]], myp = p.lam[0][kb + oy[3]];
            lf0x = cs * (mxp - m0) * rdx;
            lf0y = cs * (myp - m0) * rdy;
            lf0z = (k <= nz - 2) ? cs * (p.lam[0][own + plane] * p.rdz[k + 1] - m0 * p.rdz[k]) : T(0);
        }
        T gx = lf0x, gy = lf0y, gz = lf0z;
        T vf[NT];
#pragma unroll
        for (int f = 0; f < NT; f++) {
            const T *L = p.lam[f + 1];
            const uint8_t *B = p.branch + (long long)f * nz * plane;
            T lphi = T(0);
            // i direction: faces a = i-2 .. i+1; cell c is stencil member 3, 2, 1, 0 of them
            T lm[5];
#pragma unroll
            for (int q = 0; q < 5; q++) lm[q] = L[kb + ox[q]];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const T lF = cs * (lm[q + 1] - lm[q]) * rdx;
                const int br = B[kb + ox[q]] & 3;
                lphi += lF * mxf[q] * face_coef<T>(mxf[q] >= T(0), br, 3 - q);
            }
            // j direction
#pragma unroll
            for (int q = 0; q < 5; q++) lm[q] = L[kb + oy[q]];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const T lF = cs * (lm[q + 1] - lm[q]) * rdy;
                const int br = (B[kb + oy[q]] >> 2) & 3;
                lphi += lF * myf[q] * face_coef<T>(myf[q] >= T(0), br, 3 - q);
            }
            // k direction: faces a = k-2 .. k+1 that exist; ghost levels fold into the boundary cell
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int a = k + q - 2;
                if (a < 0 || a > nz - 2) continue;
                const T lF = cs * (L[(long long)(a + 1) * plane + ox[2]] * p.rdz[a + 1] -
                                   L[(long long)a * plane + ox[2]] * p.rdz[a]);
                const int br = (B[(long long)a * plane + ox[2]] >> 4) & 3;
                const bool u = mzf[q] >= T(0);
                T cf = T(0);
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    int cell = a + m - 1;
                    cell = cell < 0 ? 0 : (cell > nz - 1 ? nz - 1 : cell);
                    if (cell == k) cf += face_coef<T>(u, br, m);
                }
                lphi += lF * mzf[q] * cf;
            }
            // gradient of M at the cell's own faces
            const T *Y = p.ys[f + 1];
            const T *R0 = p.ys[0];
            // phi as the forward stage saw it: stored as phi in the padded
            // stage buffers, as rho*phi (converted with the reciprocal of rho) otherwise
            const bool sphi = p.ys_phi != 0;
            auto phi = [&](long long off) { return sphi ? Y[off] : Y[off] * recip(R0[off]); };
            const T ph = sphi ? Y[skb + sx[2]] : Y[skb + sx[2]] * rr;
            {
                const T mx = mxf[2];
                const T fx = face_val4<LIM>(phi(skb + sx[1]), ph, phi(skb + sx[3]), phi(skb + sx[4]), mx >= T(0));
                gx += cs * (L[kb + ox[3]] - L[own]) * rdx * fx;
                const T my = myf[2];
                const T fy = face_val4<LIM>(phi(skb + sy[1]), ph, phi(skb + sy[3]), phi(skb + sy[4]), my >= T(0));
                gy += cs * (L[kb + oy[3]] - L[own]) * rdy * fy;
                if (k <= nz - 2) {
                    const T mz = mzf[2];
                    const long long km1 = (long long)(k > 0 ? k - 1 : 0) * p.ys_plane + sx[2];
                    const long long kp1 = (long long)(k + 1) * p.ys_plane + sx[2];
                    const long long kp2 = (long long)(k + 2 < nz ? k + 2 : nz - 1) * p.ys_plane + sx[2];
                    const T fz = face_val4<LIM>(phi(km1), ph, phi(kp1), phi(kp2), mz >= T(0));
                    gz += cs * (L[own + plane] * p.rdz[k + 1] - L[own] * p.rdz[k]) * fz;
                }
            }
            vf[f] = lphi * rr;
            vrho -= lphi * ph * rr;
        }
        // gradients of the mass fluxes through the cell's own +1/2 faces
        p.gmu[own] += gx;
        p.gmv[own] += gy;
        if (k <= nz - 2) p.gmw[own + plane] += gz;
        // outputs
        T v[NF];
        v[0] = vrho;
#pragma unroll
        for (int f = 0; f < NT; f++) v[f + 1] = vf[f];
#pragma unroll
        for (int f = 0; f < NF; f++) {
            if (p.out1[0]) p.out1[f][own] = v[f];
            if (p.out2[0]) {
                T o = v[f];
                if (p.base2[0]) o += p.base2[f][own];
                if (p.add_self) o += p.lam[f][own];
                p.out2[f][own] = o;
            }
        }
    }
}

// ------------------------------------------------------------------ column transpose

// Per column: recompute the forward relaxation and sedimentation and the
// diffusion solution phi_f, then apply the transposes in reverse order:
//   diffusion:  psi = A^{-1} (rho lambda_u)  (A is symmetric),
//               lambda_x = dz psi,
//               lambda_rho_k += lambda_u phi - dz psi phi - sum over the faces of k of
//                               (dg/drho) (psi_k - psi_nb)(phi_k - phi_nb);
//   sedimentation (bottom-up):  nu_k = lambda_k + dt v w_{k-1} nu_{k-1},
//                               lambda_k = nu_k dz_k w_k,  w_k = 1/(dz_k + dt v);
//   relaxation:  lambda_rho += lambda_rhotheta r theta_ref / (1 + r),
//                lambda_rhotheta /= (1 + r).
// Scratch per column and level: m, alpha, gamma, lambda_rho increment, and
// phi and the elimination values e for every field.
template <typename T, int NF>
__global__ void __launch_bounds__(COL_TPB) adj_column_kernel(const __grid_constant__ AdjColParams<T> a) {
    constexpr int NT = NF - 1;
    constexpr int NQ = 4 + 2 * NT;
    const ColumnParams<T> &p = a.c;
    const long long ncol = p.plane, nslots = p.nslots, plane = p.plane;
    const long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nz = p.nz;
    for (long long col = slot; col < ncol; col += nslots) {
        double *sc = p.scratch + slot;
        auto S = [&](int k, int q) -> double & { return sc[(long long)(k * NQ + q) * nslots]; };
        // ---- forward: relaxation and sedimentation (in T), diffusion factorisation and solve (double)
        double g_hi = 0.0, m_up = 0.0;
        double e_up[NT];
#pragma unroll
        for (int f = 0; f < NT; f++) e_up[f] = 0.0;
        T P = T(0);
        for (int k = nz - 1; k >= 0; k--) {
            const long long o = (long long)k * plane + col;
            const T rho = p.y[0][o];
            T x[NT];
#pragma unroll
            for (int f = 0; f < NT; f++) x[f] = p.y[f + 1][o];
            if (p.do_relax) {
                T th = x[0] / rho;
                th = (th + p.relax_r * p.thref[k]) * p.relax_inv;
                x[0] = rho * th;
            }
            if (p.do_sed) {
#pragma unroll
                for (int f = 1; f < NT; f++)
                    if (f + 1 == p.sed) {
                        x[f] = (x[f] * p.dzT[k] + p.sed_dt * P) * p.sedr[k];
                        P = p.sed_v * x[f];
                    }
            }
            if (p.do_diff) {
                const double rd = to_f64(rho);
                const double g_lo = (k > 0) ? p.kc[k - 1] * (to_f64(p.y[0][o - plane]) + rd) : 0.0;
                const double b = rd * p.dz[k] + (g_lo + g_hi);
                const double t = g_hi * m_up;
                const double m = rcp_newton(fma(-g_hi, t, b));
                const double alpha = t * p.dzr_up[k];
                S(k, 0) = m;
                S(k, 1) = alpha;
                if (k < nz - 1) S(k + 1, 2) = g_hi * m * p.dzr_dn[k + 1];
#pragma unroll
                for (int f = 0; f < NT; f++) {
                    const double e = fma(alpha, e_up[f], to_f64(x[f]));
                    S(k, 4 + NT + f) = e;
                    e_up[f] = e;
                }
                g_hi = g_lo;
                m_up = m;
            }
        }
        if (p.do_diff) {
            double z[NT];
#pragma unroll
            for (int f = 0; f < NT; f++) z[f] = 0.0;
            for (int k = 0; k < nz; k++) {
                const double gk = k > 0 ? S(k, 2) : 0.0, sk = p.dz[k] * S(k, 0);
#pragma unroll
                for (int f = 0; f < NT; f++) {
                    z[f] = fma(gk, z[f], S(k, 4 + NT + f));
                    S(k, 4 + f) = sk * z[f];          // phi_f,k
                }
                S(k, 3) = 0.0;                        // lambda_rho increment
            }
            // ---- transpose of the diffusion, every field in the same sweep over k
            // (the fields' recurrences are independent, so their latencies overlap)
            double eu[NT];
#pragma unroll
            for (int f = 0; f < NT; f++) eu[f] = 0.0;
            for (int k = nz - 1; k >= 0; k--) {
                const long long o = (long long)k * plane + col;
                const double rk = to_f64(p.y[0][o]) * p.rdz64[k];   // rho_k / dz_k
                const double al = S(k, 1);
#pragma unroll
                for (int f = 0; f < NT; f++) {
                    eu[f] = fma(al, eu[f], rk * to_f64(a.lam[f + 1][o]));
                    S(k, 4 + NT + f) = eu[f];
                }
            }
            double zp[NT], psi_prev[NT], phi_prev[NT];
#pragma unroll
            for (int f = 0; f < NT; f++) zp[f] = psi_prev[f] = phi_prev[f] = 0.0;
            double carry = 0.0;   // lambda_rho increment of level k-1 still to be stored
            for (int k = 0; k < nz; k++) {
                const long long o = (long long)k * plane + col;
                const double gk = k > 0 ? S(k, 2) : 0.0, dmk = p.dz[k] * S(k, 0), kcl = k > 0 ? p.kc[k - 1] : 0.0;
                double lr = 0.0, tsum = 0.0;
#pragma unroll
                for (int f = 0; f < NT; f++) {
                    zp[f] = fma(gk, zp[f], S(k, 4 + NT + f));
                    const double psi = dmk * zp[f];
                    const double ph = S(k, 4 + f);
                    const double lu = to_f64(a.lam[f + 1][o]);
                    lr += (lu - p.dz[k] * psi) * ph;
                    tsum += kcl * (psi - psi_prev[f]) * (ph - phi_prev[f]);
                    a.lam[f + 1][o] = from_f64<T>(p.dz[k] * psi);
                    psi_prev[f] = psi;
                    phi_prev[f] = ph;
                }
                // the face k-1/2 term enters level k with a minus sign and level k-1 with a minus sign
                if (k > 0) S(k - 1, 3) = carry - tsum;
                carry = lr - tsum;
            }
            S(nz - 1, 3) = carry;
        }
        // ---- transpose of the sedimentation (bottom-up) and of the relaxation
        double nu_prev = 0.0;
        const double sv = to_f64(p.sed_v), rr = to_f64(p.relax_r), ri = to_f64(p.relax_inv);
        for (int k = 0; k < nz; k++) {
            const long long o = (long long)k * plane + col;
            if (p.do_sed) {
                double nu = to_f64(a.lam[p.sed][o]);
                if (k > 0) nu += p.dt * sv * to_f64(p.sedr[k - 1]) * nu_prev;
                nu_prev = nu;
                a.lam[p.sed][o] = from_f64<T>(nu * p.dz[k] * to_f64(p.sedr[k]));
            }
            double lrho = to_f64(a.lam[0][o]);
            if (p.do_diff) lrho += S(k, 3);
            if (p.do_relax) {
                const double lt = to_f64(a.lam[1][o]);
                lrho += lt * rr * to_f64(p.thref[k]) * ri;
                a.lam[1][o] = from_f64<T>(lt * ri);
            }
            a.lam[0][o] = from_f64<T>(lrho);
        }
    }
}

// ------------------------------------------------------------------ launchers

template <typename T, int NF, int LIM>
static cudaError_t launch_adj_stage_lim(const AdjStageParams<T> &p, cudaStream_t s) {
    dim3 block(32, 4);
    dim3 grid((p.nx + 31) / 32, (p.ny + 3) / 4);
    adj_stage_kernel<T, NF, LIM><<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename T, int NF>
static cudaError_t launch_adj_stage_nf(const AdjStageParams<T> &p, int lim, cudaStream_t s) {
    switch (lim) {
        case ASUCA_LIM_KOREN: return launch_adj_stage_lim<T, NF, ASUCA_LIM_KOREN>(p, s);
        case ASUCA_LIM_LINEAR: return launch_adj_stage_lim<T, NF, ASUCA_LIM_LINEAR>(p, s);
        case ASUCA_LIM_UPWIND1: return launch_adj_stage_lim<T, NF, ASUCA_LIM_UPWIND1>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_adj_stage(const AdjStageParams<T> &p, int nf, int lim, cudaStream_t s) {
    switch (nf) {
        case 2: return launch_adj_stage_nf<T, 2>(p, lim, s);
        case 3: return launch_adj_stage_nf<T, 3>(p, lim, s);
        case 4: return launch_adj_stage_nf<T, 4>(p, lim, s);
        case 5: return launch_adj_stage_nf<T, 5>(p, lim, s);
        case 6: return launch_adj_stage_nf<T, 6>(p, lim, s);
        case 7: return launch_adj_stage_nf<T, 7>(p, lim, s);
        case 8: return launch_adj_stage_nf<T, 8>(p, lim, s);
        case 9: return launch_adj_stage_nf<T, 9>(p, lim, s);
        case 10: return launch_adj_stage_nf<T, 10>(p, lim, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_adj_column(const AdjColParams<T> &p, int nf, int grid, cudaStream_t s) {
    switch (nf) {
#define ASUCA_ADJ_COL_CASE(N) \
        case N: adj_column_kernel<T, N><<<grid, COL_TPB, 0, s>>>(p); break;
        ASUCA_ADJ_COL_CASE(2) ASUCA_ADJ_COL_CASE(3) ASUCA_ADJ_COL_CASE(4) ASUCA_ADJ_COL_CASE(5)
        ASUCA_ADJ_COL_CASE(6) ASUCA_ADJ_COL_CASE(7) ASUCA_ADJ_COL_CASE(8) ASUCA_ADJ_COL_CASE(9)
        ASUCA_ADJ_COL_CASE(10)
#undef ASUCA_ADJ_COL_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template cudaError_t launch_adj_stage<float>(const AdjStageParams<float> &, int, int, cudaStream_t);
template cudaError_t launch_adj_stage<double>(const AdjStageParams<double> &, int, int, cudaStream_t);
template cudaError_t launch_adj_column<float>(const AdjColParams<float> &, int, int, cudaStream_t);
template cudaError_t launch_adj_column<double>(const AdjColParams<double> &, int, int, cudaStream_t);

}  // namespace asuca
