// Milne-Eddington synthesis through the instrument filters (Secs. 3.1-3.2):
// one pixel per thread, the filter/wavelength table in shared memory.
#include "common.cuh"

namespace vfisv {

// Pack filters [nf][nlam] and offsets [nlam] into the row-major table and
// append tau_k = sum_i T_k(x_i).  One block; threads stride over rows.
//
// Grid points that carry almost none of any filter's weight are left out
// (kept rows stay in grid order).  With M_k = sum_i |T_k(x_i)| and a point's
// relative weight r_i = max_k |T_k(x_i)| / M_k, the points of least r are
// dropped as long as, for every filter, the dropped |weights| sum to at most
// kMassDrop * M_k.  A filtered value S_k = sum_i T_k(x_i) y(x_i) then moves
// by at most 2^-24 M_k max|y|: the size of one FP32 rounding of a sum of that
// magnitude, so the sums are those over the whole grid to working precision.
// For the HMI-like filters (Gaussian FWHM 76 mA x sinc^2, six positions
// 69 mA apart) on the 149-point grid 63 points remain, the central
// -310 ... +310 mA; the oracle's Stokes through the cut grid differ from the
// full-grid ones by 1e-8 of the continuum.  The largest dropped set is found
// by bisection over the bit patterns of r (non-negative floats order like
// their bits).  tau_k still sums every row; a NaN or infinite weight, or a
// grid longer than kMassGrid points, keeps every row.  The number of kept
// rows goes to the last float of the tau row (as int bits).
constexpr float kMassDrop = 0x1p-24f;
constexpr int kMassGrid = 4096;
constexpr int kMassMaxNF = 128;

__global__ void pack_table_kernel(const float* __restrict__ filters, int nf,
                                  const float* __restrict__ wl, int nlam,
                                  float* __restrict__ table) {
  const int S = table_stride(nf);
  __shared__ float rbuf[kMassGrid];  // relative weight r_i of each point
  __shared__ float mass[kMassMaxNF];  // M_k
  __shared__ int wsum[32];
  __shared__ int base, lo_s, hi_s, ok_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // M_k: one warp per filter, lane-strided then a shuffle tree
  for (int k = warp; k < nf && k < kMassMaxNF; k += nw) {
    float m = 0.0f;
    for (int i = lane; i < nlam; i += 32) m += fabsf(filters[(size_t)k * nlam + i]);
    for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
    if (lane == 0) mass[k] = m;
  }
  if (threadIdx.x == 0) {
    base = 0;
    lo_s = -1;  // bits of the largest r dropped (-1: none)
    hi_s = 0;
  }
  __syncthreads();
  bool usable = nlam <= kMassGrid && nf <= kMassMaxNF;
  for (int k = 0; k < nf && usable; ++k) usable = isfinite(mass[k]);
  if (usable) {
    int rmax = 0;
    for (int i = threadIdx.x; i < nlam; i += blockDim.x) {
      float r = 0.0f;
      for (int k = 0; k < nf; ++k)
        if (mass[k] > 0.0f) r = fmaxf(r, fabsf(filters[(size_t)k * nlam + i]) / mass[k]);
      rbuf[i] = r;
      rmax = max(rmax, __float_as_int(r));
    }
    for (int o = 16; o > 0; o >>= 1) rmax = max(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    if (lane == 0) atomicMax(&hi_s, rmax);
    __syncthreads();
    // invariant: dropping r <= lo is within bounds; hi is not known to be
    for (;;) {
      const int lo = lo_s, hi = hi_s;
      if (hi - lo <= 1) break;
      const int mid = lo + (hi - lo) / 2;
      if (threadIdx.x == 0) ok_s = 1;
      __syncthreads();
      for (int k = warp; k < nf; k += nw) {
        float d = 0.0f;
        for (int i = lane; i < nlam; i += 32)
          if (__float_as_int(rbuf[i]) <= mid) d += fabsf(filters[(size_t)k * nlam + i]);
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0 && !(d <= kMassDrop * mass[k])) ok_s = 0;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        if (ok_s) lo_s = mid;
        else hi_s = mid;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  const int lo = lo_s;
  // ordered compaction, blockDim rows at a time
  for (int i0 = 0; i0 < nlam; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    const bool keep = i < nlam && (!usable || __float_as_int(rbuf[i]) > lo);
    const unsigned b = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wsum[warp] = __popc(b);
    __syncthreads();
    int off = base;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    if (keep) {
      float* row = table + (size_t)(off + __popc(b & ((1u << lane) - 1u))) * S;
      for (int k = 0; k < nf; ++k) row[k] = filters[(size_t)k * nlam + i];
      row[nf] = wl[i];
      for (int j = nf + 1; j < S; ++j) row[j] = 0.0f;
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int w = 0; w < nw; ++w) base += wsum[w];
    __syncthreads();
  }
  // tau: one warp per filter, fixed summation order (lane-strided, then a
  // shuffle tree) so the result does not depend on the launch.
  for (int k = warp; k < S; k += nw) {
    float s = 0.0f;
    if (k < nf)
      for (int i = lane; i < nlam; i += 32) s += filters[(size_t)k * nlam + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0)
      table[(size_t)nlam * S + k] = (k < nf) ? s : (k == S - 1 ? __int_as_float(base) : 0.0f);
  }
}

cudaError_t launch_pack_table(const float* filters, int nf, const float* wl, int nlam,
                              float* table, cudaStream_t s) {
  pack_table_kernel<<<1, 256, 0, s>>>(filters, nf, wl, nlam, table);
  return cudaGetLastError();
}

template <int NF>
__global__ void __launch_bounds__(128) synth_kernel(SynthArgs A) {
  extern __shared__ __align__(16) float smem[];
  const int S = table_stride(NF);
  float* tab = smem;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + table_floats(NF, A.nlam));
  if (!tma_load_table(tab, A.table, (uint32_t)(table_floats(NF, A.nlam) * sizeof(float)),
                      mbar, A.err))
    return;
  const float* tau = tab + (size_t)A.nlam * S;
  const int nl = table_rows(tab, NF, A.nlam);

  for (int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pix < A.npix;
       pix += (int64_t)gridDim.x * blockDim.x) {
    const float* p = A.params + pix * 10;
    const float B = p[0], gam = p[1], psi = p[2], eta0 = p[3], dld = p[4], dmp = p[5],
                v = p[6], S0 = p[7], S1 = p[8], alpha = p[9];
    float acc[1][4][NF];
    float accn[1][4][NF];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int k = 0; k < NF; ++k) acc[0][s][k] = accn[0][s][k] = 0.0f;
    const PixK P = make_pixk(A.lk, B, gam, eta0, dld, dmp, v);
    for (int i = 0; i < nl; ++i) {
      float T[NF];
      const float x = load_row<NF>(tab + (size_t)i * S, T);
      lambda_step<NF, false>(A.W, P, x, T, acc);
    }
    if (alpha != 1.0f) {  // non-magnetic component: the same line with B = 0
      const PixK Pn = make_pixk(A.lk, 0.0f, gam, eta0, dld, dmp, v);
      for (int i = 0; i < nl; ++i) {
        float T[NF];
        const float x = load_row<NF>(tab + (size_t)i * S, T);
        lambda_step<NF, false>(A.W, Pn, x, T, accn);
      }
    }
    float c2, s2;
    sincosf(2.0f * psi * kDeg, &s2, &c2);
    const float mus1 = A.lk.mu * S1;
    float* out = A.stokes + pix * 4 * NF;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const float yI = alpha * acc[0][0][k] + (1.0f - alpha) * accn[0][0][k];
      const float yQ = alpha * acc[0][1][k];
      const float yU = alpha * acc[0][2][k];
      const float yV = alpha * acc[0][3][k];
      out[k] = fmaf(S0, tau[k], mus1 * yI);
      out[NF + k] = mus1 * fmaf(c2, yQ, -s2 * yU);
      out[2 * NF + k] = mus1 * fmaf(s2, yQ, c2 * yU);
      out[3 * NF + k] = mus1 * yV;
    }
  }
}

template <int NF>
static cudaError_t launch_synth_nf(const SynthArgs& a, cudaStream_t s) {
  const size_t smem = table_floats(NF, a.nlam) * sizeof(float) + 16;
  auto kern = synth_kernel<NF>;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 128, smem);
  if (per < 1) per = 1;
  int64_t need = (a.npix + 127) / 128;
  int64_t grid = (int64_t)nsm * per;
  if (need < grid) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(int)grid, 128, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_synth(const SynthArgs& a, int nf, cudaStream_t s) {
  switch (nf) {
    case 1: return launch_synth_nf<1>(a, s);
    case 2: return launch_synth_nf<2>(a, s);
    case 3: return launch_synth_nf<3>(a, s);
    case 4: return launch_synth_nf<4>(a, s);
    case 5: return launch_synth_nf<5>(a, s);
    case 6: return launch_synth_nf<6>(a, s);
    case 7: return launch_synth_nf<7>(a, s);
    case 8: return launch_synth_nf<8>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace vfisv
