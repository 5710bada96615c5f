// Per-pixel preparation helpers of the paper's pipeline (Sec. 4.3): the
// empirical Stokes-I weight for full-disk maps (Eq. 14) with the continuum
// centre-to-limb variation (Eq. 15).
#include "common.cuh"

namespace vfisv {

__device__ __forceinline__ float icont_mu(float mu) {
  // Eq. 15, Horner form
  return fmaf(fmaf(fmaf(fmaf(fmaf(0.59943f, mu, -1.89979f), mu, 2.45050f), mu, -1.79238f), mu,
                   1.30590f), mu, 0.33644f);
}

__global__ void limb_weights_kernel(const float* __restrict__ obs, const float* __restrict__ mu,
                                    int64_t npix, int nf, float inv_ic0, float4 inv_sig2,
                                    float* __restrict__ w) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npix) return;
  const float* o = obs + p * 4 * nf;
  float ic = -INFINITY;
  for (int k = 0; k < nf; ++k) ic = fmaxf(ic, o[k]);
  // Eq. 14: w_I = 0.7778 |I_cont(mu) - I_cont(x,y)| + 0.3; w_Q = w_U = w_V = 1
  const float wI = fmaf(0.7778f, fabsf(icont_mu(mu[p]) - ic * inv_ic0), 0.3f);
  float* out = w + p * 4 * nf;
  for (int k = 0; k < nf; ++k) {
    out[k] = wI * wI * inv_sig2.x;
    out[nf + k] = inv_sig2.y;
    out[2 * nf + k] = inv_sig2.z;
    out[3 * nf + k] = inv_sig2.w;
  }
}

cudaError_t launch_limb_weights(const float* obs, const float* mu, int64_t npix, int nf,
                                float ic0, const float* sigma4, float* w, cudaStream_t s) {
  const float4 is2 = make_float4(1.0f / (sigma4[0] * sigma4[0]), 1.0f / (sigma4[1] * sigma4[1]),
                                 1.0f / (sigma4[2] * sigma4[2]), 1.0f / (sigma4[3] * sigma4[3]));
  limb_weights_kernel<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(obs, mu, npix, nf,
                                                                      1.0f / ic0, is2, w);
  return cudaGetLastError();
}

}  // namespace vfisv
