// One Wicker-Skamarock RK3 stage, fused (Sec. 1.1 "ASUCA on GPU"):
//   phi = (rho phi) / rho                     (one reciprocal of rho per cell)
//   face values by the Koren limiter in i, j, k, upwind by sign(M)
//   R = -[dX/dx + dY/dy + dZ/dz] + tendency,  Y_out = Y_base + cdt R
//
// Thread mapping: one thread per (i, j) column of a TX x TY tile, marching k
// upward (parallel in I/J, sequential in K).  Per level the tile's phi values
// plus a 2-wide halo in i (rows of the tile) and in j (columns of the tile)
// sit in shared memory; the corners are never needed.  The thread's own
// column keeps phi at k-1..k+2 in registers (a rolling window) and carries
// the flux through face k-1/2 from the previous level, so every vertical face
// is reconstructed once.  Periodic i/j boundaries are index wraps computed
// once per thread; threads of a ragged edge tile load wrapped cells so that
// their neighbours see the periodic values, and store nothing.
#include "common.cuh"

namespace asuca {

template <typename T, int NF, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) stage_kernel(const __grid_constant__ StageParams<T> p) {
    constexpr int NT = NF - 1;                    // fields carried as mixing ratios
    constexpr int SW = TX + 4, SH = TY + 4;
    constexpr int NHALO = 4 * (TX + TY);
    constexpr int NTHR = TX * TY;
    constexpr int MAXH = (NHALO + NTHR - 1) / NTHR;
    __shared__ T sphi[NT][SH][SW];

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const long long plane = p.plane;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int i = i0 + tx, j = j0 + ty;
    const bool valid = (i < nx) && (j < ny);
    const int ic = wrap_index(i, nx), jc = wrap_index(j, ny);
    const long long own = (long long)jc * nx + ic;
    const long long left = (long long)jc * nx + wrap_index(ic - 1, nx);
    const long long down = (long long)wrap_index(jc - 1, ny) * nx + ic;

    // halo cells served by this thread: smem slot and planar offset
    int hsx[MAXH], hsy[MAXH];
    long long hoff[MAXH];
    int nh = 0;
#pragma unroll
    for (int q = 0; q < MAXH; q++) {
        const int h = tid + q * NTHR;
        hsx[q] = 0;
        hsy[q] = 0;
        hoff[q] = 0;
        if (h < NHALO) {
            int sx, sy;
            if (h < 4 * TY) {                     // left/right halo columns
                const int r = h / 4, c = h % 4;
                sy = r + 2;
                sx = c < 2 ? c : TX + c;
            } else {                              // bottom/top halo rows
                const int h2 = h - 4 * TY;
                const int r = h2 / TX, c = h2 % TX;
                sx = c + 2;
                sy = r < 2 ? r : TY + r;
            }
            hsx[q] = sx;
            hsy[q] = sy;
            hoff[q] = (long long)wrap_index(j0 + sy - 2, ny) * nx + wrap_index(i0 + sx - 2, nx);
            nh = q + 1;
        }
    }

    // rolling window phi_{k-1}, phi_k, phi_{k+1}, phi_{k+2} (ghosts copy the boundary level)
    T win[NT][4];
    {
        const int k1 = nz > 1 ? 1 : 0, k2 = nz > 2 ? 2 : nz - 1;
        const T r0 = recip(p.yin[0][own]);
        const T r1 = recip(p.yin[0][k1 * plane + own]);
        const T r2 = recip(p.yin[0][k2 * plane + own]);
#pragma unroll
        for (int f = 0; f < NT; f++) {
            const T v0 = p.yin[f + 1][own] * r0;
            win[f][0] = v0;
            win[f][1] = v0;
            win[f][2] = p.yin[f + 1][k1 * plane + own] * r1;
            win[f][3] = p.yin[f + 1][k2 * plane + own] * r2;
        }
    }
    T zlo[NF];
#pragma unroll
    for (int f = 0; f < NF; f++) zlo[f] = T(0);

    const int lim = p.lim;
    const T rdx = p.rdx, rdy = p.rdy, cdt = p.cdt;

    for (int k = 0; k < nz; k++) {
        const long long kb = (long long)k * plane;
        // ---- fill the level-k tile: own cell from the window, halo from memory
#pragma unroll
        for (int f = 0; f < NT; f++) sphi[f][ty + 2][tx + 2] = win[f][1];
#pragma unroll
        for (int q = 0; q < MAXH; q++) {
            if (q < nh) {
                const T r = recip(p.yin[0][kb + hoff[q]]);
#pragma unroll
                for (int f = 0; f < NT; f++) sphi[f][hsy[q]][hsx[q]] = p.yin[f + 1][kb + hoff[q]] * r;
            }
        }
        __syncthreads();

        if (valid) {
            const T mup = p.mu[kb + own], mum = p.mu[kb + left];
            const T mvp = p.mv[kb + own], mvm = p.mv[kb + down];
            const bool top = (k == nz - 1);
            const T mwp = top ? T(0) : p.mw[kb + plane + own];
            const T rdz = p.rdz[k];
            const long long o = kb + own;
            {   // density: its flux is M itself
                const T r = -((mup - mum) * rdx + (mvp - mvm) * rdy + (mwp - zlo[0]) * rdz);
                zlo[0] = mwp;
                p.yout[0][o] = p.ybase[0][o] + cdt * r;
            }
            const int sx = tx + 2, sy = ty + 2;
#pragma unroll
            for (int f = 0; f < NT; f++) {
                const T c = win[f][1];
                const T xm2 = sphi[f][sy][sx - 2], xm1 = sphi[f][sy][sx - 1];
                const T xp1 = sphi[f][sy][sx + 1], xp2 = sphi[f][sy][sx + 2];
                const T ym2 = sphi[f][sy - 2][sx], ym1 = sphi[f][sy - 1][sx];
                const T yp1 = sphi[f][sy + 1][sx], yp2 = sphi[f][sy + 2][sx];
                const T xp = mup * face_value(xm1, c, xp1, xp2, mup, lim);
                const T xm = mum * face_value(xm2, xm1, c, xp1, mum, lim);
                const T yp = mvp * face_value(ym1, c, yp1, yp2, mvp, lim);
                const T ym = mvm * face_value(ym2, ym1, c, yp1, mvm, lim);
                const T zp = top ? T(0) : mwp * face_value(win[f][0], c, win[f][2], win[f][3], mwp, lim);
                T r = -((xp - xm) * rdx + (yp - ym) * rdy + (zp - zlo[f + 1]) * rdz);
                zlo[f + 1] = zp;
                if (p.tend) r += p.tend[(long long)f * nz * plane + o];
                p.yout[f + 1][o] = p.ybase[f + 1][o] + cdt * r;
            }
        }
        __syncthreads();

        // ---- advance the window: load phi at level k+3 (clamped to the top)
        if (k + 1 < nz) {
            const int kn = (k + 3 < nz) ? k + 3 : nz - 1;
            const long long on = (long long)kn * plane + own;
            const T r = recip(p.yin[0][on]);
#pragma unroll
            for (int f = 0; f < NT; f++) {
                win[f][0] = win[f][1];
                win[f][1] = win[f][2];
                win[f][2] = win[f][3];
                win[f][3] = p.yin[f + 1][on] * r;
            }
        }
    }
}

template <typename T, int NF>
static cudaError_t launch_nf(const StageParams<T> &p, cudaStream_t s) {
    constexpr int TX = 32, TY = 8;
    dim3 block(TX, TY);
    dim3 grid((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY);
    stage_kernel<T, NF, TX, TY><<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stage(const StageParams<T> &p, int nf, cudaStream_t s) {
    switch (nf) {
        case 2: return launch_nf<T, 2>(p, s);
        case 3: return launch_nf<T, 3>(p, s);
        case 4: return launch_nf<T, 4>(p, s);
        case 5: return launch_nf<T, 5>(p, s);
        case 6: return launch_nf<T, 6>(p, s);
        case 7: return launch_nf<T, 7>(p, s);
        case 8: return launch_nf<T, 8>(p, s);
        case 9: return launch_nf<T, 9>(p, s);
        case 10: return launch_nf<T, 10>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_stage<float>(const StageParams<float> &, int, cudaStream_t);
template cudaError_t launch_stage<double>(const StageParams<double> &, int, cudaStream_t);

}  // namespace asuca
