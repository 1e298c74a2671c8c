// Launcher of the HEVI acoustic short steps (acoustic.cu).
#pragma once

#include "common.cuh"

namespace asuca {

// One stage of a short step: the per-level coefficients of the stage's
// length tau, computed on the host (the base state is horizontally uniform,
// so the vertical system's matrix and its Thomas factorisation are the same
// for every column).
template <typename T>
struct AcousticParams {
    T *U, *V, *W, *S;        // the short step's start state ([nz][ny][nx]; W [nz+1][ny][nx])
    T *Uo, *Vo, *Wo, *So;    // where stage 2 writes the new state (the start state's arrays, or others)
    T *Us, *Vs, *Ws, *Ss;    // stage-1 values (workspace; Ws holds the stage-1 elimination only)
    // stage 2, when Mu is set: the mass fluxes the density equation applies,
    // (U*, V*, (1 - beta) W + beta W'), weighted by wacc, are added to (or, with
    // acc_init, stored in) Mu, Mv and the interior faces of Mw; wlo = wacc (1 - beta),
    // whi = wacc beta
    T *Mu, *Mv, *Mw;
    T wacc, wlo, whi;
    int acc_init;
    int nx, ny, nz;
    unsigned plane;
    T rdx, rdy;
    // per level k: horizontal pressure-gradient factors tau c^2 rho0_k / dx (dy),
    // tau / rho0_k, (1 - beta) / dz_k, and B_k = tau beta / (rho0_k dz_k)
    T gx[MAXNZ], gy[MAXNZ], cr[MAXNZ], cw[MAXNZ], B[MAXNZ];
    // per interior face f: (1 - beta) G_f, A_f = beta G_f (G_f = tau c^2 rho0f_f / dzc_f),
    // the lower diagonal -A_f B_{f-1}, and the factorisation: 1 / pivot_f and c'_f
    T cq[MAXNZ + 1], A[MAXNZ + 1], lo[MAXNZ + 1], inv[MAXNZ + 1], cp[MAXNZ + 1];
};

template <typename T>
cudaError_t launch_acoustic_stage(const AcousticParams<T> &p, int stage, cudaStream_t s);

// s = rho / rho0_k - 1 of every cell (the acoustic density perturbation of the
// advected density); rho0c: nz host values
template <typename T>
cudaError_t launch_hevi_init(const T *rho, const double *rho0c, T *S, int nx, int ny, int nz, cudaStream_t s);

}  // namespace asuca
