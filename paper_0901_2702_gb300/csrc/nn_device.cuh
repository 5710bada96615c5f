// Per-pixel device pieces of the initial-guess network shared by the
// training kernels (nn.cu) and the fused tensor-memory inference kernel
// (mlp_tc.cu): the activation, the continuum estimate and the decoding of the
// network outputs into an initial model.
#pragma once

#include <math.h>

#include "nn.cuh"

namespace vfisv {
namespace nn {

// GELU(x) = x Phi(x) and its derivative Phi(x) + x phi(x).
__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
  return fmaf(x, pdf, cdf);
}

// Continuum estimate: the largest of the six Stokes I samples (at least 1e-30).
__device__ __forceinline__ float ic_of(const float* o) {
  float ic = -INFINITY;
#pragma unroll
  for (int j = 0; j < 6; ++j) ic = fmaxf(ic, o[j]);
  return fmaxf(ic, 1e-30f);
}

// Network outputs y[0..10] (standardised, bias included) -> initial model
// p[0..9]; the inverse of the training targets [B, cos gamma, sin 2psi,
// cos 2psi, ln eta0, dlambdaD, a, v, S0/Ic, S1/Ic].
__device__ __forceinline__ void decode_row(const float* y, float ic, float mu,
                                           const float* out_mean, const float* out_std,
                                           float* p) {
  float t[OUT - 1];
#pragma unroll
  for (int o = 0; o < OUT - 1; ++o) t[o] = fmaf(y[o], out_std[o], out_mean[o]);
  p[0] = fmaxf(t[0], 0.0f);
  p[1] = acosf(fminf(fmaxf(t[1], -1.0f), 1.0f)) * 57.295779513082321f;
  float ps = 0.5f * atan2f(t[2], t[3]) * 57.295779513082321f;
  if (ps < 0.0f) ps += 180.0f;
  p[2] = ps;
  p[3] = expf(t[4]);
  p[4] = t[5];
  p[5] = t[6];
  p[6] = t[7];
  p[7] = t[8] * ic;
  p[8] = t[9] * ic / mu;
  p[9] = 1.0f;
}

}  // namespace nn
}  // namespace vfisv
