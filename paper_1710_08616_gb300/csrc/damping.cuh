// Launcher of the lateral and upper damping kernel (damping.cu).
#pragma once

#include "common.cuh"

namespace asuca {

constexpr int DAMP_MAXW = ASUCA_DAMP_MAX_WIDTH;

// y[f] (nf fields of the state), ref/b0/b1 ([nf][nz][ny][nx]) on the device;
// the zone and rates as asuca_damping documents them, already validated.
template <typename T>
cudaError_t launch_damping(T *const *y, int nf, const T *ref, const T *b0, const T *b1, int nx, int ny, int nz,
                           int width, int ntop, double nu_lat, double nu_top, double mtratio, double tratio,
                           double dt, int sms, cudaStream_t s);

}  // namespace asuca
