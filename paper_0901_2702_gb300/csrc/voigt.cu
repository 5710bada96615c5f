// Bulk Voigt / Faraday-Voigt evaluation (Sec. 3.2): the Weideman rational
// series used by the inversion, and the paper's Taylor-table alternative
// (Eqs. 10-13): H and F tabulated on 500 frequencies x 100 dampings and
// extrapolated from the nearest node to first or second order with the
// analytic derivatives of Eqs. 8-11.
#include "common.cuh"

namespace vfisv {

// Table geometry: u in [0, 20) with du = 0.04 (H is even and F odd in u),
// a in [0, 5) with da = 0.05.  Points outside fall back to the rational series.
constexpr int kTabU = 500, kTabA = 100;
constexpr float kTabDu = 0.04f, kTabDa = 0.05f;

__global__ void voigt_table_kernel(Weideman W, float2* __restrict__ tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kTabU * kTabA) return;
  const int ju = i % kTabU, ja = i / kTabU;
  float H, F;
  faddeeva(W, ju * kTabDu, ja * kTabDa, H, F);
  tab[i] = make_float2(H, F);
}

template <int METHOD>  // 0 rational series, 1 Taylor first order, 2 second order
__global__ void voigt_eval_kernel(Weideman W, const float2* __restrict__ tab,
                                  const float* __restrict__ a_in, const float* __restrict__ u_in,
                                  int64_t n, float* __restrict__ H_out,
                                  float* __restrict__ F_out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float a = a_in[i], u = u_in[i];
    float H, F;
    const float au = fabsf(u);
    const int ju = __float2int_rn(au * (1.0f / kTabDu));
    const int ja = __float2int_rn(a * (1.0f / kTabDa));
    if (METHOD == 0 || ju >= kTabU || ja >= kTabA || a < 0.0f) {
      faddeeva(W, u, a, H, F);
    } else {
      const float2 hf = __ldg(&tab[ja * kTabU + ju]);
      const float a0 = ja * kTabDa, u0 = ju * kTabDu;
      const float d_a = a - a0, d_u = au - u0;
      const float H0 = hf.x, F0 = hf.y;
      // Eqs. 8-9 at the node
      const float al = fmaf(2.0f * a0, H0, fmaf(2.0f * u0, F0, -kTwoInvSqrtPi));
      const float be = fmaf(2.0f * a0, F0, -2.0f * u0 * H0);
      H = fmaf(al, d_a, fmaf(be, d_u, H0));
      F = fmaf(be, d_a, fmaf(-al, d_u, F0));
      if (METHOD == 2) {  // Eqs. 12-13 (second-order terms from Eqs. 10-11)
        const float hh = fmaf(a0, al, fmaf(u0, be, H0));   // H + a alpha + u beta
        const float ff = fmaf(a0, be, fmaf(-u0, al, F0));  // F + a beta - u alpha
        const float q = fmaf(d_a, d_a, -d_u * d_u), c = 2.0f * d_a * d_u;
        H = fmaf(hh, q, fmaf(ff, c, H));
        F = fmaf(ff, q, fmaf(-hh, c, F));
      }
      if (u < 0.0f) F = -F;  // H even, F odd in u
    }
    H_out[i] = H;
    F_out[i] = F;
  }
}

size_t voigt_table_bytes() { return (size_t)kTabU * kTabA * sizeof(float2); }

cudaError_t launch_voigt_table(const Weideman& W, void* tab, cudaStream_t s) {
  voigt_table_kernel<<<(kTabU * kTabA + 255) / 256, 256, 0, s>>>(W, (float2*)tab);
  return cudaGetLastError();
}

cudaError_t launch_voigt(int method, const Weideman& W, const void* tab, const float* a,
                         const float* u, int64_t n, float* H, float* F, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = (n + 255) / 256;
  if (grid > (int64_t)nsm * 32) grid = (int64_t)nsm * 32;
  if (grid < 1) grid = 1;
  const float2* t = (const float2*)tab;
  switch (method) {
    case 0: voigt_eval_kernel<0><<<(int)grid, 256, 0, s>>>(W, t, a, u, n, H, F); break;
    case 1: voigt_eval_kernel<1><<<(int)grid, 256, 0, s>>>(W, t, a, u, n, H, F); break;
    case 2: voigt_eval_kernel<2><<<(int)grid, 256, 0, s>>>(W, t, a, u, n, H, F); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace vfisv
