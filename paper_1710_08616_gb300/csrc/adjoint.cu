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
#include <type_traits>

#include "adjoint_params.cuh"

namespace asuca {

template <typename T, int NF, int LIM>
__global__ void __launch_bounds__(256) adj_stage_kernel(const __grid_constant__ AdjStageParams<T> p) {
    constexpr int NT = NF - 1;
    // A block takes a 32 x 8 tile of cells at one level.  Per field, the
    // adjoint fluxes lambda_F M of the tile's i and j faces are formed once,
    // from tiles of lambda and the recorded branches in shared memory, and
    // every cell gathers the four faces per direction whose stencil holds it;
    // the k faces of the cell's own column are taken directly.  The face values
    // the gradient of M needs are the ones the forward stage recorded.
    constexpr int TW = 36, TH = 12, TN = TW * TH;   // tile with a halo of 2 (i: -2..33, j: -2..9)
    constexpr int NXF = 35, NYF = 11;               // i faces i0-2..i0+32 (8 rows), j faces j0-2..j0+8 (32 columns)
    __shared__ T ctab[32];
    __shared__ T sMU[TN], sMV[TN];                  // MU, MV over the tile
    __shared__ T sL[TN];                            // lambda of the current field
    __shared__ uint8_t sB[TN];                      // its branch bytes
    __shared__ T sWx[8 * NXF], sWy[NYF * 32];       // lambda_F M of the i and j faces
    __shared__ uint8_t sCx[8 * NXF], sCy[NYF * 32]; // their (upwind side, branch) as u * 4 + br
    const int lane = threadIdx.x, row = threadIdx.y, tid = row * 32 + lane;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 8, k = blockIdx.z;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int i = i0 + lane, j = j0 + row;
    const bool valid = i < nx && j < ny;
    // offsets within a field fit in 32 bits (the host checks)
    const unsigned plane = (unsigned)p.plane;
    const unsigned kb = (unsigned)k * plane;
    const bool sphi = p.ys_phi != 0;
    const T cs = p.cs, rdx = p.rdx, rdy = p.rdy;
    if (tid < 32) ctab[tid] = face_coef<T>((tid >> 4) != 0, (tid >> 2) & 3, tid & 3);
    // the tile cells this thread loads
    constexpr int PER = (TN + 255) / 256;
    unsigned to[PER];
#pragma unroll
    for (int q = 0; q < PER; q++) {
        const int c = tid + q * 256;
        to[q] = 0;
        if (c < TN) {
            const int ii = wrap_index(i0 - 2 + c % TW, nx), jj = wrap_index(j0 - 2 + c / TW, ny);
            to[q] = kb + (unsigned)(jj * nx + ii);
        }
    }
#pragma unroll
    for (int q = 0; q < PER; q++) {
        const int c = tid + q * 256;
        if (c < TN) {
            sMU[c] = p.mu[to[q]];
            sMV[c] = p.mv[to[q]];
        }
    }
    const int cc = (row + 2) * TW + lane + 2;       // the thread's cell in the tile
    const unsigned col = (unsigned)(j * nx + i);
    const unsigned own = kb + col;
    const unsigned sown = (unsigned)k * (unsigned)p.ys_plane +
                          (unsigned)((j + p.ys_oy) * p.ys_pitch + (i + p.ys_ox) * p.ys_xs);
    // the cell's own column: k faces a = k-2 .. k+1
    T mzf[4];
    T rr = T(1);
    if (valid) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int a = k + q - 2;
            mzf[q] = (a >= 0 && a <= nz - 2) ? p.mw[(unsigned)(a + 1) * plane + col] : T(0);
        }
        rr = recip(p.ys[0][sown]);
    }
    __syncthreads();
    T gx = T(0), gy = T(0), gz = T(0), vrho = T(0);
    const size_t fs = (size_t)nz * plane, ds = (size_t)NT * fs;

    // tiles of lambda and the branch bytes of field f, loaded into registers one
    // field ahead so that the loads overlap the previous field's work
    T nL[PER];
    uint8_t nB[PER];
    auto fetch = [&](int f) {
        const T *L = p.lam[f + 1];
        const uint8_t *B = p.branch + (size_t)f * fs;
#pragma unroll
        for (int q = 0; q < PER; q++) {
            const int c = tid + q * 256;
            if (c < TN) {
                nL[q] = L[to[q]];
                nB[q] = B[to[q]];
            }
        }
    };
    fetch(0);
    for (int f = 0; f < NT; f++) {
        const T *L = p.lam[f + 1];
        const uint8_t *B = p.branch + (size_t)f * fs;
#pragma unroll
        for (int q = 0; q < PER; q++) {
            const int c = tid + q * 256;
            if (c < TN) {
                sL[c] = nL[q];
                sB[c] = nB[q];
            }
        }
        __syncthreads();
        if (f + 1 < NT) fetch(f + 1);
        // ---- lambda_F M of the tile's faces, once each
        for (int t = tid; t < 8 * NXF + NYF * 32; t += 256) {
            if (t < 8 * NXF) {          // i face a = i0 - 2 + x at row r (cells x, x+1 of tile row r+2)
                const int r = t / NXF, x = t % NXF, c = (r + 2) * TW + x;
                const T m = sMU[c];
                sWx[t] = cs * (sL[c + 1] - sL[c]) * rdx * m;
                sCx[t] = (uint8_t)((m >= T(0) ? 4 : 0) | (sB[c] & 3));
            } else {                    // j face b = j0 - 2 + y at column x (cells y, y+1 of tile column x+2)
                const int t2 = t - 8 * NXF, y = t2 / 32, x = t2 % 32, c = y * TW + x + 2;
                const T m = sMV[c];
                sWy[t2] = cs * (sL[c + TW] - sL[c]) * rdy * m;
                sCy[t2] = (uint8_t)((m >= T(0) ? 4 : 0) | ((sB[c] >> 2) & 3));
            }
        }
        __syncthreads();
        if (valid) {
            T lphi = T(0);
            // i direction: faces a = i-2 .. i+1 (tile face index lane .. lane+3); c is member 3-q
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int t = row * NXF + lane + q;
                lphi += sWx[t] * ctab[sCx[t] * 4 + (3 - q)];
            }
            // j direction
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int t = (row + q) * 32 + lane;
                lphi += sWy[t] * ctab[sCy[t] * 4 + (3 - q)];
            }
            // k direction: faces a = k-2 .. k+1 that exist; next to a lid the ghost
            // levels fold several stencil members into the boundary cell
            T lz[5];
#pragma unroll
            for (int q = 0; q < 5; q++) {
                const int lev = k + q - 2;
                lz[q] = (lev >= 0 && lev < nz) ? L[(unsigned)lev * plane + col] : T(0);
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int a = k + q - 2;
                if (a < 0 || a > nz - 2) continue;
                const T lF = cs * (lz[q + 1] * p.rdz[a + 1] - lz[q] * p.rdz[a]);
                const int br = (B[(unsigned)a * plane + col] >> 4) & 3;
                const T *ct = ctab + (mzf[q] >= T(0) ? 16 : 0) + br * 4;
                T cf;
                if (a >= 1 && a + 2 <= nz - 1) {
                    cf = ct[3 - q];
                } else {
                    cf = T(0);
#pragma unroll
                    for (int m = 0; m < 4; m++) {
                        int cell = a + m - 1;
                        cell = cell < 0 ? 0 : (cell > nz - 1 ? nz - 1 : cell);
                        if (cell == k) cf += ct[m];
                    }
                }
                lphi += lF * mzf[q] * cf;
            }
            // gradient of M at the cell's own faces, this field's share, with the
            // recorded face values
            const T *Y = p.ys[f + 1];
            const T ph = sphi ? Y[sown] : Y[sown] * rr;
            const T *fv = p.facev + (size_t)f * fs + own;
            gx += cs * (sL[cc + 1] - sL[cc]) * rdx * fv[0];
            gy += cs * (sL[cc + TW] - sL[cc]) * rdy * fv[ds];
            if (k <= nz - 2) gz += cs * (lz[3] * p.rdz[k + 1] - lz[2] * p.rdz[k]) * fv[2 * ds];
            // the field's output
            const T v = lphi * rr;
            if (p.out1[0]) p.out1[f + 1][own] = v;
            if (p.out2[0]) {
                T o = v;
                if (p.base2[0]) o += p.base2[f + 1][own];
                if (p.add_self) o += lz[2];
                p.out2[f + 1][own] = o;
            }
            vrho -= lphi * ph * rr;
        }
        __syncthreads();   // the tiles are reloaded for the next field
    }
    // ---- density: its output and its terms of the gradients of the cell's own faces
    if (valid) {
        const T m0 = p.lam[0][own];
        gx += cs * (p.lam[0][kb + (unsigned)(j * nx + wrap_index(i + 1, nx))] - m0) * rdx;
        gy += cs * (p.lam[0][kb + (unsigned)(wrap_index(j + 1, ny) * nx + i)] - m0) * rdy;
        if (k <= nz - 2) gz += cs * (p.lam[0][own + plane] * p.rdz[k + 1] - m0 * p.rdz[k]);
        p.gmu[own] += gx;
        p.gmv[own] += gy;
        if (k <= nz - 2) p.gmw[own + plane] += gz;
        if (p.out1[0]) p.out1[0][own] = vrho;
        if (p.out2[0]) {
            T o = vrho;
            if (p.base2[0]) o += p.base2[0][own];
            if (p.add_self) o += m0;
            p.out2[0][own] = o;
        }
    }
}

// ------------------------------------------------------------------ column transpose

// Per column, the transposes of the column pass in reverse order:
//   diffusion:  psi = A^{-1} (rho lambda_u)  (A is symmetric),
//               lambda_x = dz psi,
//               lambda_rho_k += lambda_u phi - dz psi phi - sum over the faces of k of
//                               (dg/drho) (psi_k - psi_nb)(phi_k - phi_nb);
//   sedimentation (bottom-up):  nu_k = lambda_k + dt v w_{k-1} nu_{k-1},
//                               lambda_k = nu_k dz_k w_k,  w_k = 1/(dz_k + dt v);
//   relaxation:  lambda_rho += lambda_rhotheta r theta_ref / (1 + r),
//                lambda_rhotheta /= (1 + r).
// The factorisation of A (m, alpha, gamma per level, with the scaled
// unknowns of the forward pass) and the forward solution (z per field, phi
// = dz m z) come from the record the forward column pass of the same step
// left (ColumnParams::rec), so only the transposed solve runs here.
// A block takes 32 columns (the lanes) and one warp per field (rho*theta and
// each tracer): the warp of field f runs the transposed solve, writes the
// field's adjoint and leaves its share of the lambda_rho increment per level
// in the scratch; then the warps, dealt levels round-robin, add the shares to
// lambda_rho in field order (a fixed order, so the result does not depend on
// scheduling).  Both sweeps run in double in both precisions.  With float
// fields the arithmetic around them is float, as in the forward step: the
// right-hand side rho lambda / dz is formed in float and widened, and the
// lambda_rho shares are products of the double differences rounded to float
// once.  Scratch per column and level: per field the elimination value
// (reused for the field's lambda_rho share), and the relaxation share.
template <typename T, int NF>
__global__ void __launch_bounds__(32 * (NF - 1)) adj_column_kernel(const __grid_constant__ AdjColParams<T> a) {
    constexpr int NT = NF - 1;
    constexpr int NQ = 3 + 2 * NT;
    constexpr int NR = NF + 2;                      // record entries per level: m, alpha, gamma, z[NT]
    constexpr bool F32 = std::is_same<T, float>::value;
    const ColumnParams<T> &p = a.c;
    const int lane = threadIdx.x, f = threadIdx.y;   // f: field f + 1 of the state
    const long long plane = p.plane;
    const size_t pl = (size_t)plane;
    const long long nslots = (long long)gridDim.x * 32;
    const int nz = p.nz;
    double *const sc = p.scratch + (long long)blockIdx.x * 32 + lane;
#define S(k, q) sc[(long long)((k) * NQ + (q)) * nslots]
    const int qe = 3 + f, qr = 3 + NT;               // this field's elimination / share slot; relaxation share
    const bool is_th = f == 0, is_sed = p.do_sed && (f + 1 == p.sed);
    const T *R = p.y[0];
    T *lam = a.lam[f + 1];
    const double sv = to_f64(p.sed_v), rr = to_f64(p.relax_r), ri = to_f64(p.relax_inv);

    for (long long c0 = (long long)blockIdx.x * 32; c0 < plane; c0 += nslots) {
        const long long col = c0 + lane;
        const bool valid = col < plane;
        const double *rc = p.rec + col;
#define RC(k, q) rc[(size_t)((k) * NR + (q)) * pl]
        __syncthreads();   // the previous group's shares have been added
        if (valid) {
            if (p.do_diff) {
                // transpose of the diffusion: elimination top-down on rho lambda / dz
                double eu = 0.0;
                long long o = (long long)(nz - 1) * plane + col;
                double al = RC(nz - 1, 1);
                T r = R[o], l = lam[o];
                for (int k = nz - 1; k >= 0; k--, o -= plane) {
                    double al_n = 0.0;
                    T r_n = T(0), l_n = T(0);
                    if (k > 0) {
                        al_n = RC(k - 1, 1);
                        r_n = R[o - plane];
                        l_n = lam[o - plane];
                    }
                    double rhs;
                    if constexpr (F32) rhs = to_f64(r * p.rdzT[k] * l);
                    else rhs = to_f64(r) * p.rdz64[k] * to_f64(l);
                    eu = fma(al, eu, rhs);
                    S(k, qe) = eu;
                    al = al_n;
                    r = r_n;
                    l = l_n;
                }
            }
            // bottom-up: transposed back substitution, the field's lambda_rho
            // shares, then the sedimentation and relaxation transposes
            double zp = 0.0, psi_prev = 0.0, phi_prev = 0.0;
            double gk = 0.0, ek = 0.0, mk = 0.0, zk = 0.0;
            if (p.do_diff) {
                ek = S(0, qe);
                mk = RC(0, 0);
                zk = RC(0, 3 + f);
            }
            T lk = lam[col];
            long long o = col;
            if constexpr (F32) {
                float carry = 0.f, nu_prev = 0.f;
                const float svf = p.sed_v, rrf = p.relax_r, rif = p.relax_inv, dtf = p.sed_dt;
                for (int k = 0; k < nz; k++, o += plane) {
                    double gn = 0.0, en = 0.0, mn = 0.0, zn = 0.0;
                    T ln = T(0);
                    if (k + 1 < nz) {
                        if (p.do_diff) {
                            gn = RC(k + 1, 2);
                            en = S(k + 1, qe);
                            mn = RC(k + 1, 0);
                            zn = RC(k + 1, 3 + f);
                        }
                        ln = lam[o + plane];
                    }
                    float lout;
                    bool write = false;
                    if (p.do_diff) {
                        const double sk = p.dz[k] * mk;
                        zp = fma(gk, zp, ek);
                        const double psi = sk * zp;
                        const double ph = sk * zk;
                        // A = (lambda_u - dz psi) phi, B = (dg/drho)(psi - psi_prev)(phi - phi_prev)
                        const float A = d2f_bits(fma(-p.dz[k], psi, to_f64(lk))) * d2f_bits(ph);
                        const float B = k > 0 ? p.kcT[k - 1] * d2f_bits(psi - psi_prev) * d2f_bits(ph - phi_prev) : 0.f;
                        // level k-1 takes A - B(k-1/2) - B(k+1/2); the last one now
                        if (k > 0) S(k - 1, qe) = f2d_bits_any(carry - B);
                        carry = A - B;
                        psi_prev = psi;
                        phi_prev = ph;
                        lout = p.dzT[k] * d2f_bits(psi);
                        write = true;
                    } else {
                        lout = lk;
                    }
                    if (is_sed) {
                        float nu = lout;
                        if (k > 0) nu += dtf * svf * p.sedr[k - 1] * nu_prev;
                        nu_prev = nu;
                        lout = nu * p.dzT[k] * p.sedr[k];
                        write = true;
                    }
                    if (is_th && p.do_relax) {
                        S(k, qr) = f2d_bits_any(lout * rrf * p.thref[k] * rif);   // relaxation share
                        lout = lout * rif;
                        write = true;
                    }
                    if (write) lam[o] = lout;
                    gk = gn;
                    ek = en;
                    mk = mn;
                    zk = zn;
                    lk = ln;
                }
                if (p.do_diff) S(nz - 1, qe) = f2d_bits_any(carry);
            } else {
                double carry = 0.0, nu_prev = 0.0;
                for (int k = 0; k < nz; k++, o += plane) {
                    double gn = 0.0, en = 0.0, mn = 0.0, zn = 0.0;
                    T ln = T(0);
                    if (k + 1 < nz) {
                        if (p.do_diff) {
                            gn = RC(k + 1, 2);
                            en = S(k + 1, qe);
                            mn = RC(k + 1, 0);
                            zn = RC(k + 1, 3 + f);
                        }
                        ln = lam[o + plane];
                    }
                    double lout;
                    bool write = false;
                    if (p.do_diff) {
                        const double kcl = k > 0 ? p.kc[k - 1] : 0.0;
                        const double sk = p.dz[k] * mk;
                        zp = fma(gk, zp, ek);
                        const double psi = sk * zp;
                        const double ph = sk * zk;
                        const double lu = to_f64(lk);
                        const double A = (lu - p.dz[k] * psi) * ph;
                        const double B = kcl * (psi - psi_prev) * (ph - phi_prev);   // face k-1/2
                        // level k-1 takes A - B(k-1/2) - B(k+1/2); the last one now
                        if (k > 0) S(k - 1, qe) = carry - B;
                        carry = A - B;
                        psi_prev = psi;
                        phi_prev = ph;
                        lout = to_f64(from_f64<T>(p.dz[k] * psi));
                        write = true;
                    } else {
                        lout = to_f64(lk);
                    }
                    if (is_sed) {
                        double nu = lout;
                        if (k > 0) nu += p.dt * sv * to_f64(p.sedr[k - 1]) * nu_prev;
                        nu_prev = nu;
                        lout = to_f64(from_f64<T>(nu * p.dz[k] * to_f64(p.sedr[k])));
                        write = true;
                    }
                    if (is_th && p.do_relax) {
                        S(k, qr) = lout * rr * to_f64(p.thref[k]) * ri;   // relaxation share of lambda_rho
                        lout = lout * ri;
                        write = true;
                    }
                    if (write) lam[o] = from_f64<T>(lout);
                    gk = gn;
                    ek = en;
                    mk = mn;
                    zk = zn;
                    lk = ln;
                }
                if (p.do_diff) S(nz - 1, qe) = carry;
            }
        }
#undef RC
        __syncthreads();
        // ---- lambda_rho, levels dealt to the warps
        if (valid) {
            for (int k = f; k < nz; k += NT) {
                const long long o = (long long)k * plane + col;
                if constexpr (F32) {
                    float lrho = a.lam[0][o];
                    if (p.do_diff) {
                        float inc = 0.f;
#pragma unroll
                        for (int q = 0; q < NT; q++) inc += d2f_bits(S(k, 3 + q));
                        lrho += inc;
                    }
                    if (p.do_relax) lrho += d2f_bits(S(k, qr));
                    a.lam[0][o] = lrho;
                } else {
                    double lrho = to_f64(a.lam[0][o]);
                    if (p.do_diff) {
                        double inc = 0.0;
#pragma unroll
                        for (int q = 0; q < NT; q++) inc += S(k, 3 + q);
                        lrho += inc;
                    }
                    if (p.do_relax) lrho += S(k, qr);
                    a.lam[0][o] = from_f64<T>(lrho);
                }
            }
        }
    }
#undef S
}

// ------------------------------------------------------------------ launchers

template <typename T, int NF, int LIM>
static cudaError_t launch_adj_stage_lim(const AdjStageParams<T> &p, cudaStream_t s) {
    dim3 block(32, 8);
    dim3 grid((p.nx + 31) / 32, (p.ny + 7) / 8, p.nz);
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
        case N: adj_column_kernel<T, N><<<grid, dim3(32, N - 1), 0, s>>>(p); break;
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
