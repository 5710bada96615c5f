// Mixed NN-initialised inversion: after the LM run from the network's guess,
// pixels that did not converge or whose chi2 exceeds a threshold are flagged,
// gathered and inverted again from the standard guess; the better of the two
// results (lower chi2) is kept.  The flagged count stays on the device.
// With confidence routing, pixels whose confidence output (the network's
// estimate of its own log squared error) is above a threshold skip the LM
// run from the guess: they are flagged from the start and take the plain
// run's result.
#include "common.cuh"
#include "nn.cuh"

namespace vfisv {
namespace nn {

__global__ void flag_gather_kernel(const int32_t* __restrict__ status,
                                   const float* __restrict__ chi2, int64_t npix,
                                   float chi2_flag, bool flag_unconverged,
                                   const float* __restrict__ obs,
                                   const float* __restrict__ w, int64_t w_stride, int nobs,
                                   unsigned long long* __restrict__ count,
                                   int64_t* __restrict__ index, float* __restrict__ obs_g,
                                   float* __restrict__ w_g, int32_t* __restrict__ flagged) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npix) return;
  const int st = status[p];
  const bool conv = (st == VFISV_PIX_CONVERGED || st == VFISV_PIX_STALLED);
  const bool f = (st != VFISV_PIX_BAD_INPUT) &&
                 ((flag_unconverged && !conv) || !(chi2[p] <= chi2_flag));
  if (flagged) flagged[p] = f ? 1 : 0;
  if (!f) return;
  const int64_t j = (int64_t)atomicAdd(count, 1ull);
  index[j] = p;
  for (int o = 0; o < nobs; ++o) obs_g[j * nobs + o] = obs[p * nobs + o];
  if (w_g)
    for (int o = 0; o < nobs; ++o) w_g[j * nobs + o] = w[p * w_stride + o];
}

cudaError_t flag_and_gather(const int32_t* status, const float* chi2, int64_t npix,
                            float chi2_flag, bool flag_unconverged, const float* obs,
                            const float* w,
                            int64_t w_stride, int nobs, int64_t* count, int64_t* index,
                            float* obs_g, float* w_g, int32_t* flagged, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int64_t), s);
  if (e != cudaSuccess) return e;
  const unsigned nb = (unsigned)((npix + 255) / 256);
  flag_gather_kernel<<<nb, 256, 0, s>>>(status, chi2, npix, chi2_flag, flag_unconverged, obs, w,
                                        w_stride, nobs,
                                        (unsigned long long*)count, index, obs_g, w_g, flagged);
  return cudaGetLastError();
}

// Routing by the confidence output: pixels with conf > conf_route get an
// empty first-stage result (status NAN_STATE, chi2 = +inf, no iterations,
// the network's guess as parameters), which the flag step re-inverts and the
// merge replaces; the others are listed for the first-stage LM run (one
// atomic per warp, so the list keeps the pixel order within each warp).
__global__ void route_kernel(const float* __restrict__ conf, int64_t npix, float conf_route,
                             const float* __restrict__ init, int64_t* __restrict__ list,
                             unsigned long long* __restrict__ count, float* __restrict__ params,
                             float* __restrict__ chi2, int32_t* __restrict__ iters,
                             int32_t* __restrict__ status) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = p < npix;
  // a NaN confidence is routed too (the guess cannot be trusted)
  const bool routed = in && !(conf[p] <= conf_route);
  const unsigned keep = __ballot_sync(0xffffffffu, in && !routed);
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (keep) {
    if (lane == __ffs(keep) - 1) base = atomicAdd(count, (unsigned long long)__popc(keep));
    base = __shfl_sync(0xffffffffu, base, __ffs(keep) - 1);
  }
  if (!in) return;
  if (routed) {
    for (int q = 0; q < 10; ++q) params[p * 10 + q] = init[p * 10 + q];
    chi2[p] = INFINITY;
    iters[p] = 0;
    status[p] = VFISV_PIX_NAN_STATE;
  } else {
    list[base + __popc(keep & ((1u << lane) - 1u))] = p;
  }
}

cudaError_t route_by_confidence(const float* conf, int64_t npix, float conf_route,
                                const float* init, int64_t* list, int64_t* count, float* params,
                                float* chi2, int32_t* iters, int32_t* status, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int64_t), s);
  if (e != cudaSuccess) return e;
  const unsigned nb = (unsigned)((npix + 255) / 256);
  route_kernel<<<nb, 256, 0, s>>>(conf, npix, conf_route, init, list,
                                  (unsigned long long*)count, params, chi2, iters, status);
  return cudaGetLastError();
}

__device__ __forceinline__ void merge_one(int64_t j, int lane, const int64_t* __restrict__ index,
                                          const float* __restrict__ p2, const float* __restrict__ c2,
                                          const int32_t* __restrict__ i2,
                                          const int32_t* __restrict__ s2,
                                          const float* __restrict__ cov2, float* __restrict__ params,
                                          float* __restrict__ chi2, int32_t* __restrict__ iters,
                                          int32_t* __restrict__ status, float* __restrict__ cov) {
  const int64_t p = index[j];
  int act = 0;  // 1: take the plain result, 2: no valid result (zero covariance)
  if (lane == 0) {
    iters[p] += i2[j];
    const int sp = s2[j];
    const bool plain_ok = (sp != VFISV_PIX_NAN_STATE) && isfinite(c2[j]);
    const bool nn_ok = (status[p] != VFISV_PIX_NAN_STATE) && isfinite(chi2[p]);
    if (plain_ok && (!nn_ok || c2[j] < chi2[p])) {
      for (int q = 0; q < 10; ++q) params[p * 10 + q] = p2[j * 10 + q];
      chi2[p] = c2[j];
      status[p] = sp;
      act = 1;
    } else if (status[p] == VFISV_PIX_NAN_STATE) {
      // no valid result from either run (a routed pixel's row was never written)
      act = 2;
    }
  }
  act = __shfl_sync(0xffffffffu, act, 0);
  if (!cov || act == 0) return;
  for (int q = lane; q < 100; q += 32)
    cov[p * 100 + q] = (act == 1 && cov2) ? cov2[j * 100 + q] : 0.0f;
}

// One warp per re-inverted pixel: lane 0 takes the decision, the warp copies
// the 100-float covariance row with coalesced loads and stores.
__global__ void merge_kernel(const int64_t* __restrict__ count, const int64_t* __restrict__ index,
                             const float* __restrict__ p2, const float* __restrict__ c2,
                             const int32_t* __restrict__ i2, const int32_t* __restrict__ s2,
                             const float* __restrict__ cov2, float* __restrict__ params,
                             float* __restrict__ chi2, int32_t* __restrict__ iters,
                             int32_t* __restrict__ status, float* __restrict__ cov) {
  const int lane = threadIdx.x & 31;
  const int64_t n = *count;
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += stride)
    merge_one(j, lane, index, p2, c2, i2, s2, cov2, params, chi2, iters, status, cov);
}

cudaError_t merge_plain(const int64_t* count, const int64_t* index, int64_t npix_max,
                        const float* p2, const float* c2, const int32_t* i2, const int32_t* s2,
                        const float* cov2, float* params, float* chi2, int32_t* iters,
                        int32_t* status, float* cov, cudaStream_t s) {
  int64_t nb = (npix_max * 32 + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;  // grid-stride over the device-side count
  if (nb < 1) nb = 1;
  merge_kernel<<<(unsigned)nb, 256, 0, s>>>(count, index, p2, c2, i2, s2, cov2, params, chi2, iters,
                                            status, cov);
  return cudaGetLastError();
}

}  // namespace nn
}  // namespace vfisv
