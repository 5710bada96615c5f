// Wide-instrument path: inputs sampled by many narrow instrument profiles
// over a fine synthesis grid (spectrograph-shaped data, e.g. 112 samples x 4
// Stokes parameters from 448 grid points), where the filter-position kernels'
// register accumulators (rows x Stokes x filters per thread) cannot hold the
// whole convolution.  One pixel per warp:
//   1. the fine grid is walked in chunks of 64 points; each lane evaluates
//      two points (synthesis and, for the inversion, the six Jacobian rows
//      of Secs. 3-4, the same per-point arithmetic as the filter kernels)
//      into a per-warp shared-memory buffer;
//   2. each lane owns the samples k = lane + 32 j and adds the chunk's
//      points inside its instrument band (at most 32 points) to them;
//   3. the inversion forms chi2 (Eq. 1, FP64) and, after an accepted step,
//      J^T W J and J^T W r from the owned samples, reduced across the warp;
//   4. lane 0 runs the FP64 damped solve (Eqs. 4-5) and the Table 2 rule.
// The instrument table is compacted on the device into bands (first point,
// length, weights) and staged in shared memory with one TMA bulk copy.
#include "common.cuh"
#include "solve.cuh"

namespace vfisv {

constexpr int kWMaxF = 128;          // samples per Stokes parameter
constexpr int kWBand = 32;           // fine points per instrument profile
constexpr int kWMaxLam = 1024;       // fine grid points
constexpr int kWChunk = 64;          // fine points per chunk: two per lane
constexpr int kWOwn = kWMaxF / 32;   // samples owned by a lane
constexpr int kWPad = 29;            // row pitch of the chunk buffer (28 values + 1)
constexpr int kWWarps = 4;           // pixels in flight per CTA
constexpr int kWBandStride = kWBand + 4;  // [lo, n, tau, pad, w[32]] per sample

// Shared-memory layout of the compacted table: bands [nf][kWBandStride], then
// the fine grid x[nlam], padded to a multiple of 4 floats (16-byte TMA size).
__host__ __device__ inline int wide_table_floats(int nf, int nlam) {
  return ((nf * kWBandStride + nlam) + 3) & ~3;
}

__global__ void wide_pack_kernel(const float* __restrict__ filters, int nf,
                                 const float* __restrict__ wl, int nlam,
                                 float* __restrict__ table, int* __restrict__ err) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = warp; k < nf; k += blockDim.x >> 5) {
    const float* row = filters + (size_t)k * nlam;
    // first and last non-zero point; tau in a fixed order (lane-strided
    // partial sums, then a shuffle tree)
    int lo = nlam, hi = -1;
    float s = 0.0f;
    for (int i = lane; i < nlam; i += 32) {
      const float t = row[i];
      if (t != 0.0f) {
        lo = min(lo, i);
        hi = max(hi, i);
      }
      s += t;
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    const int n = (hi >= lo) ? hi - lo + 1 : 0;
    float* b = table + (size_t)k * kWBandStride;
    if (lane == 0) {
      if (n > kWBand) atomicExch(err, VFISV_E_UNSUPPORTED);
      b[0] = __int_as_float(n > 0 ? lo : 0);
      b[1] = __int_as_float(min(n, kWBand));
      b[2] = s;
      b[3] = 0.0f;
    }
    b[4 + lane] = (lane < n && lane < kWBand) ? row[lo + lane] : 0.0f;
  }
  for (int i = threadIdx.x; i < nlam; i += blockDim.x) table[(size_t)nf * kWBandStride + i] = wl[i];
  const int tot = wide_table_floats(nf, nlam);
  for (int i = nf * kWBandStride + nlam + threadIdx.x; i < tot; i += blockDim.x) table[i] = 0.0f;
}

// Filtered rows of one pixel: acc[j][r][s] = sum_i T_k(x_i) y_r,s(x_i) for the
// owned samples k = lane + 32 j (rows r: Stokes, then with DERIV the six
// Jacobian rows before their per-pixel scale factors).
template <bool DERIV>
__device__ __forceinline__ void wide_pass(const Weideman& W, const PixK& P, const float* tab,
                                          int nf, int nlam, float* vbuf, int lane,
                                          float (&acc)[kWOwn][DERIV ? kRows : 1][4]) {
  constexpr int R = DERIV ? kRows : 1;
#pragma unroll
  for (int j = 0; j < kWOwn; ++j)
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int s = 0; s < 4; ++s) acc[j][r][s] = 0.0f;
  const float* xg = tab + nf * kWBandStride;
#pragma unroll 1
  for (int c0 = 0; c0 < nlam; c0 += kWChunk) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int li = lane + 32 * t, i = c0 + li;
      if (i < nlam) {
        float v[R][4][1];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int s = 0; s < 4; ++s) v[r][s][0] = 0.0f;
        const float one[1] = {1.0f};
        lambda_step<1, DERIV>(W, P, xg[i], one, v);
        float* dst = vbuf + li * kWPad;
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int s = 0; s < 4; ++s) dst[r * 4 + s] = v[r][s][0];
      }
    }
    __syncwarp();
    const int c1 = min(c0 + kWChunk, nlam);
#pragma unroll
    for (int j = 0; j < kWOwn; ++j) {
      const int k = lane + 32 * j;
      if (k < nf) {
        const float* b = tab + k * kWBandStride;
        const int lo = __float_as_int(b[0]), n = __float_as_int(b[1]);
        const int i0 = max(lo, c0), i1 = min(lo + n, c1);
#pragma unroll 1
        for (int i = i0; i < i1; ++i) {
          const float w = b[4 + (i - lo)];
          const float* src = vbuf + (i - c0) * kWPad;
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int s = 0; s < 4; ++s) acc[j][r][s] = fmaf(w, src[r * 4 + s], acc[j][r][s]);
        }
      }
    }
    __syncwarp();
  }
}

struct WideSynthArgs {
  const float* params;
  int64_t npix;
  const float* table;
  int nf, nlam;
  float* stokes;
  int* err;
  Weideman W;
  LineK lk;
};

__global__ void __launch_bounds__(32 * kWWarps) wide_synth_kernel(WideSynthArgs A) {
  extern __shared__ __align__(16) float smem[];
  const int tabf = wide_table_floats(A.nf, A.nlam);
  float* tab = smem;
  float* vbufs = smem + tabf;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(vbufs + kWWarps * kWChunk * kWPad + 2);
  if (!tma_load_table(tab, A.table, (uint32_t)(tabf * sizeof(float)), mbar, A.err)) return;
  if (*A.err) return;  // a band wider than the kernel takes
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* vbuf = vbufs + warp * kWChunk * kWPad;
  const int nf = A.nf;
  for (int64_t pix = (int64_t)blockIdx.x * kWWarps + warp; pix < A.npix;
       pix += (int64_t)gridDim.x * kWWarps) {
    const float* p = A.params + pix * 10;
    const float B = p[0], gam = p[1], psi = p[2], eta0 = p[3], dld = p[4], dmp = p[5],
                v = p[6], S0 = p[7], S1 = p[8], alpha = p[9];
    float acc[kWOwn][1][4], accn[kWOwn][1][4];
    wide_pass<false>(A.W, make_pixk(A.lk, B, gam, eta0, dld, dmp, v), tab, nf, A.nlam, vbuf,
                     lane, acc);
    if (alpha != 1.0f) {  // non-magnetic component: the same line with B = 0
      wide_pass<false>(A.W, make_pixk(A.lk, 0.0f, gam, eta0, dld, dmp, v), tab, nf, A.nlam,
                       vbuf, lane, accn);
    } else {
#pragma unroll
      for (int j = 0; j < kWOwn; ++j)
#pragma unroll
        for (int s = 0; s < 4; ++s) accn[j][0][s] = 0.0f;
    }
    float c2, s2;
    sincosf(2.0f * psi * kDeg, &s2, &c2);
    const float mus1 = A.lk.mu * S1;
    float* out = A.stokes + pix * 4 * nf;
#pragma unroll
    for (int j = 0; j < kWOwn; ++j) {
      const int k = lane + 32 * j;
      if (k < nf) {
        const float tau = tab[k * kWBandStride + 2];
        const float yI = alpha * acc[j][0][0] + (1.0f - alpha) * accn[j][0][0];
        const float yQ = alpha * acc[j][0][1], yU = alpha * acc[j][0][2];
        const float yV = alpha * acc[j][0][3];
        out[k] = fmaf(S0, tau, mus1 * yI);
        out[nf + k] = mus1 * fmaf(c2, yQ, -s2 * yU);
        out[2 * nf + k] = mus1 * fmaf(s2, yQ, c2 * yU);
        out[3 * nf + k] = mus1 * yV;
      }
    }
  }
}

// Warp-wide sum: every lane gets the total (fixed butterfly order).
__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Per-warp LM state in shared memory (written by lane 0, read by all).
struct WideWarpState {
  float A[kScratchPerSlot];  // packed J^T W J and J^T W r at the best model
  float M[10], Mt[10];
  double chi2b, eps;
  long long pix;
  int it;
};

__global__ void __launch_bounds__(32 * kWWarps, 1) wide_invert_kernel(InvertArgs A, int nf) {
  extern __shared__ __align__(16) float smem[];
  const int tabf = wide_table_floats(nf, A.nlam);
  float* tab = smem;
  float* vbufs = smem + tabf;
  WideWarpState* states =
      reinterpret_cast<WideWarpState*>(vbufs + kWWarps * kWChunk * kWPad + 2);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(states + kWWarps);
  if (!tma_load_table(tab, A.table, (uint32_t)(tabf * sizeof(float)), mbar, A.err)) return;
  if (*A.err) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* vbuf = vbufs + warp * kWChunk * kWPad;
  WideWarpState& S = states[warp];
  const int nobs = 4 * nf;
  const int dof = nobs - A.nfree;
  const int64_t npix = A.npix_dev ? *A.npix_dev : A.npix;
  const float mu = A.lk.mu;

  if (lane == 0) S.pix = -1;
  __syncwarp();
  while (true) {
    bool fresh = false;
    if (S.pix < 0) {
      long long pix = 0;
      if (lane == 0) pix = (long long)atomicAdd(A.queue, 1ull);
      pix = __shfl_sync(0xffffffffu, pix, 0);
      if (pix >= npix) break;
      fresh = true;
      const float* o = A.obs + pix * nobs;
      const float* wv = weight_row(A, pix, nobs);
      bool bad = false;
      float wsum = 0.0f, ic = -INFINITY;
      for (int j = lane; j < nobs; j += 32) {
        const float ov = o[j], ww = wv[j];
        bad |= !isfinite(ov) || !isfinite(ww);
        wsum += isfinite(ww) ? ww : 0.0f;
        if (j < nf) ic = fmaxf(ic, isfinite(ov) ? ov : 0.0f);
      }
      bad = __any_sync(0xffffffffu, bad);
      wsum = warp_sum(wsum);
      for (int o2 = 16; o2 > 0; o2 >>= 1) ic = fmaxf(ic, __shfl_xor_sync(0xffffffffu, ic, o2));
      bad |= !(wsum > 0.0f);
      if (lane == 0) {
        float Mt[10];
        if (A.init) {
          const float guess[10] = {500.f, 60.f, 45.f, 10.f, 35.f, 0.25f, 0.f, 0.25f, 0.75f, 1.f};
          for (int j = 0; j < 10; ++j) {
            const float v = A.init[pix * 10 + j];
            bad |= !isfinite(v);
            Mt[j] = isfinite(v) ? v : guess[j];
          }
        } else {
          Mt[0] = 500.f; Mt[1] = 60.f; Mt[2] = 45.f; Mt[3] = 10.f; Mt[4] = 35.f;
          Mt[5] = 0.25f; Mt[6] = 0.f;
          Mt[7] = 0.25f * ic;
          Mt[8] = 0.75f * ic / mu;
        }
        Mt[9] = 1.0f;
        apply_bounds(Mt);
        for (int j = 0; j < 10; ++j) S.Mt[j] = Mt[j];
        S.it = 0;
        S.eps = A.eps0;
        S.pix = pix;
      }
      bad = __shfl_sync(0xffffffffu, (int)bad, 0) != 0;
      __syncwarp();
      if (bad) {
        if (lane < 10) A.params_out[pix * 10 + lane] = S.Mt[lane];
        if (lane == 0) {
          A.chi2_out[pix] = 0.0f;
          A.iters_out[pix] = 0;
          A.status_out[pix] = VFISV_PIX_BAD_INPUT;
          map_retired(A, pix);
        }
        if (A.cov_out)
          for (int j = lane; j < 100; j += 32) A.cov_out[pix * 100 + j] = 0.0f;
        if (lane == 0) S.pix = -1;
        __syncwarp();
        continue;
      }
    } else {
      if (lane == 0) {
        double d[kNP];
        damped_step_fp64(S.A, 1, A.free_mask, S.eps, d);
        float Mt[10];
        for (int j = 0; j < kNP; ++j) Mt[j] = (float)((double)S.M[j] + d[j]);
        Mt[9] = 1.0f;
        apply_bounds(Mt);
        for (int j = 0; j < 10; ++j) S.Mt[j] = Mt[j];
      }
      __syncwarp();
    }

    // ---- fused synthesis + Jacobian at the trial model ----
    float Mt[10];
#pragma unroll
    for (int j = 0; j < 10; ++j) Mt[j] = S.Mt[j];
    float acc[kWOwn][kRows][4];
    wide_pass<true>(A.W, make_pixk(A.lk, Mt[0], Mt[1], Mt[3], Mt[4], Mt[5], Mt[6]), tab, nf,
                    A.nlam, vbuf, lane, acc);
    const long long pix = S.pix;
    const float* o = A.obs + pix * nobs;
    const float* wv = weight_row(A, pix, nobs);
    float c2p, s2p;
    sincosf(2.0f * Mt[2] * kDeg, &s2p, &c2p);
    const float mus1 = mu * Mt[8];
    const float s0 = Mt[7];
    // ---- chi2 (Eq. 1, FP64) ----
    double c2l = 0.0;
#pragma unroll
    for (int j = 0; j < kWOwn; ++j) {
      const int k = lane + 32 * j;
      if (k < nf) {
        const float tau = tab[k * kWBandStride + 2];
        const float q0 = acc[j][0][1], u0 = acc[j][0][2];
        const float syn[4] = {fmaf(s0, tau, mus1 * acc[j][0][0]), mus1 * fmaf(c2p, q0, -s2p * u0),
                              mus1 * fmaf(s2p, q0, c2p * u0), mus1 * acc[j][0][3]};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const double r = (double)(o[s * nf + k] - syn[s]);
          c2l = fma((double)wv[s * nf + k] * r, r, c2l);
        }
      }
    }
    const double c2 = warp_sum(c2l) / (double)dof;

    // ---- accept / converge (uniform across the warp) ----
    bool accept, retire = false;
    int status = VFISV_PIX_MAXITER;
    int it = S.it;
    if (fresh) {
      accept = isfinite(c2);
      if (!accept) {
        retire = true;
        status = VFISV_PIX_NAN_STATE;
      }
    } else {
      ++it;
      const double chi2b = S.chi2b;
      accept = isfinite(c2) && c2 < chi2b;
      const double eps_used = S.eps;
      const double eps = eps_update(eps_used, accept);
      if (accept) {
        const double rel = (chi2b - c2) / chi2b;
        if (rel < A.conv_rtol && eps_used <= A.conv_eps) {
          retire = true;
          status = VFISV_PIX_CONVERGED;
        }
      } else if (eps >= 1e12) {
        retire = true;
        status = VFISV_PIX_STALLED;
      }
      __syncwarp();
      if (lane == 0) S.eps = eps;
    }

    if (accept) {
      // ---- J^T W J and J^T W r at the new best model ----
      constexpr int rowOf[kNP] = {kRowB, kRowG, -1, kRowE, kRowD, kRowA, kRowV, -1, -1};
      const RowScale Rs = row_scale(A.lk, Mt[3], Mt[4]);
      float a[kNPk], g[kNP];
#pragma unroll
      for (int i = 0; i < kNPk; ++i) a[i] = 0.0f;
#pragma unroll
      for (int i = 0; i < kNP; ++i) g[i] = 0.0f;
#pragma unroll
      for (int j = 0; j < kWOwn; ++j) {
        const int k = lane + 32 * j;
        if (k < nf) {
          const float tau = tab[k * kWBandStride + 2];
          const float q0 = acc[j][0][1], u0 = acc[j][0][2];
          const float Qk = mus1 * fmaf(c2p, q0, -s2p * u0);
          const float Uk = mus1 * fmaf(s2p, q0, c2p * u0);
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const int sa = (s == 0) ? 0 : (s == 3 ? 3 : 1);
            const int sb = (s == 0) ? 0 : (s == 3 ? 3 : 2);
            const float cA = (s == 1) ? c2p : (s == 2 ? s2p : 1.0f);
            const float cB = (s == 1) ? -s2p : (s == 2 ? c2p : 0.0f);
            float J[kNP];
#pragma unroll
            for (int p = 0; p < kNP; ++p)
              if (rowOf[p] >= 0)
                J[p] = (mus1 * Rs.s[rowOf[p]]) *
                       fmaf(cA, acc[j][rowOf[p]][sa], cB * acc[j][rowOf[p]][sb]);
            J[2] = (s == 1) ? -2.0f * kDeg * Uk : (s == 2 ? 2.0f * kDeg * Qk : 0.0f);
            J[7] = (s == 0) ? tau : 0.0f;
            const float lin = fmaf(cA, acc[j][0][sa], cB * acc[j][0][sb]);
            J[8] = mu * lin;
            const float sv = (s == 0) ? fmaf(s0, tau, mus1 * lin) : mus1 * lin;
            const float ww = wv[s * nf + k];
            const float rr = o[s * nf + k] - sv;
#pragma unroll
            for (int p = 0; p < kNP; ++p) {
              const float wj = ww * J[p];
              g[p] = fmaf(wj, rr, g[p]);
#pragma unroll
              for (int q = 0; q <= p; ++q) a[tri(p, q)] = fmaf(wj, J[q], a[tri(p, q)]);
            }
          }
        }
      }
#pragma unroll
      for (int i = 0; i < kNPk; ++i) a[i] = warp_sum(a[i]);
#pragma unroll
      for (int i = 0; i < kNP; ++i) g[i] = warp_sum(g[i]);
      __syncwarp();
      if (lane == 0) {
        for (int i = 0; i < kNPk; ++i) S.A[i] = a[i];
        for (int i = 0; i < kNP; ++i) S.A[kNPk + i] = g[i];
        for (int j = 0; j < 10; ++j) S.M[j] = Mt[j];
        S.chi2b = c2;
      }
      __syncwarp();
    }
    if (!retire && it >= A.max_iter) retire = true;
    __syncwarp();
    if (lane == 0) S.it = it;
    __syncwarp();

    if (retire) {
      if (lane == 0) {
        double chi2b = S.chi2b;
        float Mo[10];
        for (int j = 0; j < 10; ++j) Mo[j] = (status == VFISV_PIX_NAN_STATE) ? S.Mt[j] : S.M[j];
        if (status == VFISV_PIX_NAN_STATE) chi2b = c2;
        for (int j = 0; j < 10; ++j) A.params_out[pix * 10 + j] = Mo[j];
        A.chi2_out[pix] = (float)chi2b;
        A.iters_out[pix] = it;
        A.status_out[pix] = status;
        if (A.cov_out) {
          float* cv = A.cov_out + pix * 100;
          if (status == VFISV_PIX_NAN_STATE) {
            for (int j = 0; j < 100; ++j) cv[j] = 0.0f;
          } else {
            covariance_fp64(S.A, 1, A.free_mask, cv, false);
          }
        }
        map_retired(A, pix);
        S.pix = -1;
      }
      __syncwarp();
    }
  }
}

size_t wide_table_bytes(int nf, int nlam) { return (size_t)wide_table_floats(nf, nlam) * 4; }

static size_t wide_smem(int nf, int nlam, bool invert) {
  size_t b = (size_t)wide_table_floats(nf, nlam) * 4 + (size_t)kWWarps * kWChunk * kWPad * 4 + 8;
  if (invert) b += kWWarps * sizeof(WideWarpState);
  return ((b + 15) & ~(size_t)15) + 16;
}

bool wide_supported(int nf, int nlam) {
  return nf >= 1 && nf <= kWMaxF && nlam >= 1 && nlam <= kWMaxLam;
}

cudaError_t launch_wide_pack(const float* filters, int nf, const float* wl, int nlam,
                             float* table, int* err, cudaStream_t s) {
  wide_pack_kernel<<<1, 256, 0, s>>>(filters, nf, wl, nlam, table, err);
  return cudaGetLastError();
}

static int wide_grid(const void* kern, size_t smem, int64_t npix) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * kWWarps, smem);
  if (per < 1) per = 1;
  int64_t g = (int64_t)nsm * per;
  const int64_t need = (npix + kWWarps - 1) / kWWarps;
  if (need < g) g = need;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_wide_synth(const float* params, int64_t npix, const float* table, int nf,
                              int nlam, float* stokes, int* err, const Weideman& W,
                              const LineK& lk, cudaStream_t s) {
  const size_t smem = wide_smem(nf, nlam, false);
  cudaError_t e = cudaFuncSetAttribute(wide_synth_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  WideSynthArgs a{params, npix, table, nf, nlam, stokes, err, W, lk};
  wide_synth_kernel<<<wide_grid((const void*)wide_synth_kernel, smem, npix), 32 * kWWarps, smem,
                      s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_wide_invert(const InvertArgs& a, int nf, cudaStream_t s) {
  const size_t smem = wide_smem(nf, a.nlam, true);
  cudaError_t e = cudaFuncSetAttribute(wide_invert_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  wide_invert_kernel<<<wide_grid((const void*)wide_invert_kernel, smem, a.npix), 32 * kWWarps,
                       smem, s>>>(a, nf);
  return cudaGetLastError();
}

}  // namespace vfisv
