// Wide-instrument path: inputs sampled by many narrow instrument profiles
// over a fine synthesis grid (spectrograph-shaped data, e.g. 112 samples x 4
// Stokes parameters from 448 grid points), where the filter-position kernels'
// register accumulators (rows x Stokes x filters per thread) cannot hold the
// whole convolution.  One pixel per warp:
//   1. the fine grid is walked in chunks of 64 points; each lane evaluates
//      two points (synthesis and, for the inversion, the six Jacobian rows
//      of Secs. 3-4, the same per-point arithmetic as the filter kernels)
//      into a per-warp shared-memory buffer;
//   2. the samples whose instrument band (at most 32 points) meets the chunk
//      are spread over the lanes, which add the chunk's points to per-warp
//      shared accumulators with float4 reads of the transposed chunk;
//   3. the inversion forms chi2 (Eq. 1; compensated FP32 partial sums,
//      combined and compared in FP64) and, after an accepted step, J^T W J
//      and J^T W r, reduced across the warp;
//   4. the FP64 damped solve (Eqs. 4-5) runs spread over the warp's lanes;
//      the covariance is left to the batched covariance kernel.
// The instrument table is compacted on the device into bands (first point,
// length, weights) and staged in shared memory with one TMA bulk copy.
#include "common.cuh"
#include "solve.cuh"

namespace vfisv {

constexpr int kWMaxF = 128;          // samples per Stokes parameter
constexpr int kWBand = 32;           // fine points per instrument profile
constexpr int kWMaxLam = 1024;       // fine grid points
constexpr int kWChunk = 64;          // fine points per chunk: two per lane
constexpr int kWMaxChunks = kWMaxLam / kWChunk;
constexpr int kWWarps = 4;           // pixels in flight per CTA
constexpr int kWBand4 = kWBand + 4;  // a band starting on a multiple of 4, padded to 4
constexpr int kWBandStride = kWBand4 + 4;  // [lo4, n4, tau, pad, w[36]] per sample

// Compacted table: bands [nf][kWBandStride], the active sample range of each
// chunk [kWMaxChunks][2] (int), then the fine grid x[nlam]; padded to a
// multiple of 4 floats (16-byte TMA size).
__host__ __device__ inline int wide_chunks_at(int nf) { return nf * kWBandStride; }
__host__ __device__ inline int wide_x_at(int nf) { return nf * kWBandStride + 2 * kWMaxChunks; }
__host__ __device__ inline int wide_table_floats(int nf, int nlam) {
  return (wide_x_at(nf) + nlam + 3) & ~3;
}

__global__ void wide_pack_kernel(const float* __restrict__ filters, int nf,
                                 const float* __restrict__ wl, int nlam,
                                 float* __restrict__ table, int* __restrict__ err) {
  __shared__ int slo[kWMaxF], shi[kWMaxF];
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
    if (n > kWBand && lane == 0) atomicExch(err, VFISV_E_UNSUPPORTED);
    // the band starts on a multiple of 4 (aligned float4 reads) and its
    // length is padded to a multiple of 4 with the zeros around it
    const int lo4 = (n > 0) ? (lo & ~3) : 0;
    const int n4 = (n > 0 && n <= kWBand) ? ((hi - lo4 + 1) + 3) & ~3 : 0;
    float* b = table + (size_t)k * kWBandStride;
    if (lane == 0) {
      b[0] = __int_as_float(lo4);
      b[1] = __int_as_float(n4);
      b[2] = s;
      b[3] = 0.0f;
      slo[k] = lo4;
      shi[k] = lo4 + n4;  // exclusive
    }
    for (int t = lane; t < kWBand4; t += 32)
      b[4 + t] = (t < n4 && lo4 + t < nlam) ? row[lo4 + t] : 0.0f;
  }
  __syncthreads();
  // samples whose band meets each chunk: [first, last] (their hull)
  int* ch = reinterpret_cast<int*>(table + wide_chunks_at(nf));
  for (int c = warp; c < kWMaxChunks; c += blockDim.x >> 5) {
    const int c0 = c * kWChunk, c1 = c0 + kWChunk;
    int kf = 1 << 30, kl = -1;
    for (int k = lane; k < nf; k += 32)
      if (slo[k] < c1 && shi[k] > c0 && shi[k] > slo[k]) {
        kf = min(kf, k);
        kl = max(kl, k);
      }
    for (int o = 16; o > 0; o >>= 1) {
      kf = min(kf, __shfl_xor_sync(0xffffffffu, kf, o));
      kl = max(kl, __shfl_xor_sync(0xffffffffu, kl, o));
    }
    if (lane == 0) {
      ch[2 * c] = (kl >= 0) ? kf : 0;
      ch[2 * c + 1] = kl;
    }
  }
  for (int i = threadIdx.x; i < nlam; i += blockDim.x) table[wide_x_at(nf) + i] = wl[i];
  const int tot = wide_table_floats(nf, nlam);
  for (int i = wide_x_at(nf) + nlam + threadIdx.x; i < tot; i += blockDim.x) table[i] = 0.0f;
}

// Filtered rows of one pixel into the warp's shared accumulators
// accs[k * P + v], P = 4 R + 1, for every sample k (rows r: Stokes, then
// with DERIV the six Jacobian rows before their per-pixel scale factors;
// v = 4 r + Stokes).  vbuf holds one chunk transposed, [4 R][kWChunk].
template <bool DERIV>
__device__ __forceinline__ void wide_pass(const Weideman& W, const PixK& P, const float* tab,
                                          int nf, int nlam, float* vbuf, float* accs, int lane) {
  constexpr int R = DERIV ? kRows : 1;
  constexpr int NV = 4 * R, PA = NV + 1;
  for (int t = lane; t < nf * PA; t += 32) accs[t] = 0.0f;
  const float* xg = tab + wide_x_at(nf);
  const int* ch = reinterpret_cast<const int*>(tab + wide_chunks_at(nf));
  __syncwarp();
#pragma unroll 1
  for (int c0 = 0, c = 0; c0 < nlam; c0 += kWChunk, ++c) {
#pragma unroll 1
    for (int t = 0; t < 2; ++t) {
      const int li = lane + 32 * t, i = c0 + li;
      float v[R][4][1];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) v[r][s][0] = 0.0f;
      if (i < nlam) {
        const float one[1] = {1.0f};
        lambda_step<1, DERIV>(W, P, xg[i], one, v);
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) vbuf[(r * 4 + s) * kWChunk + li] = v[r][s][0];
    }
    __syncwarp();
    const int c1 = min(c0 + kWChunk, nlam);
    const int kf = ch[2 * c], kl = ch[2 * c + 1];
#pragma unroll 1
    for (int k = kf + lane; k <= kl; k += 32) {
      const float* b = tab + k * kWBandStride;
      const int lo4 = __float_as_int(b[0]), n4 = __float_as_int(b[1]);
      const int i0 = max(lo4, c0), i1 = min(lo4 + n4, (c1 + 3) & ~3);
      if (i0 >= i1) continue;
      float a[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) a[q] = 0.0f;
#pragma unroll 1
      for (int i = i0; i < i1; i += 4) {
        const float4 w = *reinterpret_cast<const float4*>(b + 4 + (i - lo4));
        const int col = i - c0;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const float4 x = *reinterpret_cast<const float4*>(vbuf + q * kWChunk + col);
          a[q] = fmaf(w.x, x.x, fmaf(w.y, x.y, fmaf(w.z, x.z, fmaf(w.w, x.w, a[q]))));
        }
      }
      float* dst = accs + k * PA;
#pragma unroll
      for (int q = 0; q < NV; ++q) dst[q] += a[q];
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

// Shared memory of a CTA: the table, then per warp the chunk buffer
// [4R][kWChunk] and the accumulators [nf][4R + 1] (twice for synthesis: the
// magnetic and the non-magnetic component), then per warp the LM state.
__host__ __device__ inline int wide_warp_floats(int nf, bool deriv) {
  const int nv = deriv ? 4 * kRows : 4;
  const int acc = nf * (nv + 1) * (deriv ? 1 : 2);
  return ((nv * kWChunk + acc) + 3) & ~3;
}

__global__ void __launch_bounds__(32 * kWWarps) wide_synth_kernel(WideSynthArgs A) {
  extern __shared__ __align__(16) float smem[];
  const int tabf = wide_table_floats(A.nf, A.nlam);
  const int wf = wide_warp_floats(A.nf, false);
  float* tab = smem;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + tabf + kWWarps * wf);
  if (!tma_load_table(tab, A.table, (uint32_t)(tabf * sizeof(float)), mbar, A.err)) return;
  if (*A.err) return;  // a band wider than the kernel takes
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nf = A.nf;
  float* vbuf = smem + tabf + warp * wf;
  float* acc = vbuf + 4 * kWChunk;
  float* accn = acc + nf * 5;
  for (int64_t pix = (int64_t)blockIdx.x * kWWarps + warp; pix < A.npix;
       pix += (int64_t)gridDim.x * kWWarps) {
    const float* p = A.params + pix * 10;
    const float B = p[0], gam = p[1], psi = p[2], eta0 = p[3], dld = p[4], dmp = p[5],
                v = p[6], S0 = p[7], S1 = p[8], alpha = p[9];
    wide_pass<false>(A.W, make_pixk(A.lk, B, gam, eta0, dld, dmp, v), tab, nf, A.nlam, vbuf,
                     acc, lane);
    if (alpha != 1.0f)  // non-magnetic component: the same line with B = 0
      wide_pass<false>(A.W, make_pixk(A.lk, 0.0f, gam, eta0, dld, dmp, v), tab, nf, A.nlam,
                       vbuf, accn, lane);
    float c2, s2;
    sincosf(2.0f * psi * kDeg, &s2, &c2);
    const float mus1 = A.lk.mu * S1;
    float* out = A.stokes + pix * 4 * nf;
    for (int k = lane; k < nf; k += 32) {
      const float tau = tab[k * kWBandStride + 2];
      const float* a = acc + k * 5;
      const float In = (alpha != 1.0f) ? accn[k * 5] : 0.0f;
      const float yI = alpha * a[0] + (1.0f - alpha) * In;
      const float yQ = alpha * a[1], yU = alpha * a[2], yV = alpha * a[3];
      out[k] = fmaf(S0, tau, mus1 * yI);
      out[nf + k] = mus1 * fmaf(c2, yQ, -s2 * yU);
      out[2 * nf + k] = mus1 * fmaf(s2, yQ, c2 * yU);
      out[3 * nf + k] = mus1 * yV;
    }
    __syncwarp();
  }
}

// Warp-wide sum: every lane gets the total (fixed butterfly order, the same
// on every lane because addition commutes).
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

// The damped step of Eqs. 4-5 in FP64, spread over the warp.  An FP64
// instruction holds an SMSP's FP64 pipe ~80 cycles whatever the number of
// active lanes, so one lane solving alone (~600 instructions) would cost
// more than the wavelength pass; here lane l holds packed elements l and
// l + 32 of the Jacobi-scaled matrix and the factorisation, the two
// substitutions and the unscaling take ~130 FP64 instructions.  The
// factorisation and the forward substitution apply the same operations in
// the same order per element as the one-lane Cholesky (right-looking
// updates in increasing k) and give identical results; the back
// substitution accumulates its terms in the opposite order.
// Returns false (uniformly) when a pivot is not comfortably positive; the
// caller then runs the one-lane path with its eigen-decomposition fallback.
__device__ __forceinline__ void tri_ij(int e, int& i, int& j) {
  i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= e) ++i;
  while (i * (i + 1) / 2 > e) --i;
  j = e - i * (i + 1) / 2;
}

__device__ __forceinline__ double shfl_d(double v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}

// element e of the packed matrix from its owner lane (e & 31, register e >> 5)
__device__ __forceinline__ double fetch(double m0, double m1, int e) {
  const double a = shfl_d(m0, e & 31), b = shfl_d(m1, e & 31);
  return (e >> 5) ? b : a;
}

__device__ bool warp_damped_step(const float* Ash, uint32_t free_mask, double eps, int lane,
                                 double* delta /* shared [9] */) {
  int i0, j0, i1, j1;
  tri_ij(lane, i0, j0);
  const bool has1 = lane + 32 < kNPk;
  tri_ij(has1 ? lane + 32 : 0, i1, j1);
  // Jacobi scaling
  double sc = 0.0;
  bool held = true;
  if (lane < kNP) {
    const double d = (double)Ash[tri(lane, lane)];
    held = !((free_mask >> lane) & 1u) || !(d > 0.0) || !isfinite(d);
    sc = held ? 0.0 : rsqrt(d);
  }
  const uint32_t hmask = __ballot_sync(0xffffffffu, lane < kNP && held);
  // every lane runs the shuffles of both slots (uniform control flow)
  const double si0 = shfl_d(sc, i0), sj0 = shfl_d(sc, j0);
  const double si1 = shfl_d(sc, i1), sj1 = shfl_d(sc, j1);
  double m0, m1 = 0.0;
  {
    const bool hi = (hmask >> i0) & 1u, hj = (hmask >> j0) & 1u;
    m0 = (i0 == j0) ? (hi ? 1.0 : 1.0 + eps) : ((hi || hj) ? 0.0 : (double)Ash[lane] * si0 * sj0);
  }
  if (has1) {
    const bool hi = (hmask >> i1) & 1u, hj = (hmask >> j1) & 1u;
    m1 = (i1 == j1) ? (hi ? 1.0 : 1.0 + eps)
                    : ((hi || hj) ? 0.0 : (double)Ash[lane + 32] * si1 * sj1);
  }
  double b = 0.0;  // right-hand side on lanes 0..8
  if (lane < kNP && !((hmask >> lane) & 1u)) b = (double)Ash[kNPk + lane] * sc;
  double rown = 0.0;  // reciprocal pivot of row `lane`
  // right-looking factorisation
#pragma unroll 1
  for (int j = 0; j < kNP; ++j) {
    const int ejj = tri(j, j);
    const double p = shfl_d((ejj >> 5) ? m1 : m0, ejj & 31);
    if (!(p > 1e-10)) return false;
    const double r = rsqrt(p);
    if (lane == j) rown = r;
    // column j below the diagonal
    if (j0 == j && i0 > j) m0 *= r;
    if (has1 && j1 == j && i1 > j) m1 *= r;
    // trailing update of elements (i, k), i >= k > j
    const double lij0 = fetch(m0, m1, tri(max(i0, j), j)), lkj0 = fetch(m0, m1, tri(max(j0, j), j));
    const double lij1 = fetch(m0, m1, tri(max(i1, j), j)), lkj1 = fetch(m0, m1, tri(max(j1, j), j));
    if (j0 > j) m0 = fma(-lij0, lkj0, m0);
    if (has1 && j1 > j) m1 = fma(-lij1, lkj1, m1);
  }
  // forward substitution L y = b (b_i on lane i)
#pragma unroll 1
  for (int i = 0; i < kNP; ++i) {
    if (lane == i) b *= rown;
    const double yi = shfl_d(b, i);
    const double lmi = fetch(m0, m1, tri(max(lane, i), min(lane, i)));
    if (lane > i && lane < kNP) b = fma(-lmi, yi, b);
  }
  // back substitution L^T x = y
#pragma unroll 1
  for (int i = kNP - 1; i >= 0; --i) {
    if (lane == i) b *= rown;
    const double xi = shfl_d(b, i);
    const double lim = fetch(m0, m1, tri(max(lane, i), min(lane, i)));
    if (lane < i) b = fma(-lim, xi, b);
  }
  if (lane < kNP) delta[lane] = ((hmask >> lane) & 1u) ? 0.0 : sc * b;
  __syncwarp();
  return true;
}

// Per-warp LM state in shared memory (written by lane 0, read by all).
struct WideWarpState {
  float A[kScratchPerSlot];  // packed J^T W J and J^T W r at the best model
  float M[10], Mt[10];
  double delta[kNP];
  double chi2b, eps;
  long long pix;
  int it;
};

__global__ void __launch_bounds__(32 * kWWarps, 1) wide_invert_kernel(InvertArgs A, int nf) {
  extern __shared__ __align__(16) float smem[];
  const int tabf = wide_table_floats(nf, A.nlam);
  const int wf = wide_warp_floats(nf, true);
  float* tab = smem;
  WideWarpState* states = reinterpret_cast<WideWarpState*>(smem + tabf + kWWarps * wf);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(states + kWWarps);
  if (!tma_load_table(tab, A.table, (uint32_t)(tabf * sizeof(float)), mbar, A.err)) return;
  if (*A.err) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* vbuf = smem + tabf + warp * wf;
  float* accs = vbuf + 4 * kRows * kWChunk;
  constexpr int PA = 4 * kRows + 1;
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
        __syncwarp();
        if (lane == 0) S.pix = -1;
        __syncwarp();
        continue;
      }
    } else {
      // ---- damped step (Eqs. 4-5), FP64 over the warp ----
      const double eps = S.eps;
      const bool ok = warp_damped_step(S.A, A.free_mask, eps, lane, S.delta);
      if (lane == 0) {
        double d[kNP];
        if (ok) {
          for (int j = 0; j < kNP; ++j) d[j] = S.delta[j];
        } else {
          damped_step_fp64(S.A, 1, A.free_mask, eps, d);  // with the eigen fallback
        }
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
    wide_pass<true>(A.W, make_pixk(A.lk, Mt[0], Mt[1], Mt[3], Mt[4], Mt[5], Mt[6]), tab, nf,
                    A.nlam, vbuf, accs, lane);
    const long long pix = S.pix;
    const float* o = A.obs + pix * nobs;
    const float* wv = weight_row(A, pix, nobs);
    float c2p, s2p;
    sincosf(2.0f * Mt[2] * kDeg, &s2p, &c2p);
    const float mus1 = mu * Mt[8];
    const float s0 = Mt[7];
    // ---- chi2 (Eq. 1): compensated FP32 partial sums per lane (TwoProduct
    // and TwoSum: exact to ~1e-14 relative for a lane's few terms), combined
    // and compared in FP64 ----
    double c2l;
    {
      float qs = 0.0f, qc = 0.0f;
#pragma unroll 1
      for (int k = lane; k < nf; k += 32) {
        const float tau = tab[k * kWBandStride + 2];
        const float* a = accs + k * PA;
        const float q0 = a[1], u0 = a[2];
        const float syn[4] = {fmaf(s0, tau, mus1 * a[0]), mus1 * fmaf(c2p, q0, -s2p * u0),
                              mus1 * fmaf(s2p, q0, c2p * u0), mus1 * a[3]};
#pragma unroll
        for (int st = 0; st < 4; ++st) {
          const float r = o[st * nf + k] - syn[st];
          const float wr = wv[st * nf + k] * r;
          const float ew = fmaf(wv[st * nf + k], r, -wr);  // wr + ew = w r exactly
          const float p = wr * r;
          const float ep = fmaf(wr, r, -p) + ew * r;
          const float t = qs + p;
          const float bp = t - qs;
          qc += ((qs - (t - bp)) + (p - bp)) + ep;
          qs = t;
        }
      }
      c2l = (double)qs + (double)qc;
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
      float am[kNPk], g[kNP];
#pragma unroll
      for (int i = 0; i < kNPk; ++i) am[i] = 0.0f;
#pragma unroll
      for (int i = 0; i < kNP; ++i) g[i] = 0.0f;
#pragma unroll 1
      for (int k = lane; k < nf; k += 32) {
        const float tau = tab[k * kWBandStride + 2];
        const float* a = accs + k * PA;
        const float q0 = a[1], u0 = a[2];
        const float Qk = mus1 * fmaf(c2p, q0, -s2p * u0);
        const float Uk = mus1 * fmaf(s2p, q0, c2p * u0);
#pragma unroll 1
        for (int st = 0; st < 4; ++st) {
          const int sa = (st == 0) ? 0 : (st == 3 ? 3 : 1);
          const int sb = (st == 0) ? 0 : (st == 3 ? 3 : 2);
          const float cA = (st == 1) ? c2p : (st == 2 ? s2p : 1.0f);
          const float cB = (st == 1) ? -s2p : (st == 2 ? c2p : 0.0f);
          float J[kNP];
#pragma unroll
          for (int pp = 0; pp < kNP; ++pp)
            if (rowOf[pp] >= 0)
              J[pp] = (mus1 * Rs.s[rowOf[pp]]) *
                      fmaf(cA, a[rowOf[pp] * 4 + sa], cB * a[rowOf[pp] * 4 + sb]);
          J[2] = (st == 1) ? -2.0f * kDeg * Uk : (st == 2 ? 2.0f * kDeg * Qk : 0.0f);
          J[7] = (st == 0) ? tau : 0.0f;
          const float lin = fmaf(cA, a[sa], cB * a[sb]);
          J[8] = mu * lin;
          const float sv = (st == 0) ? fmaf(s0, tau, mus1 * lin) : mus1 * lin;
          const float ww = wv[st * nf + k];
          const float rr = o[st * nf + k] - sv;
#pragma unroll
          for (int pp = 0; pp < kNP; ++pp) {
            const float wj = ww * J[pp];
            g[pp] = fmaf(wj, rr, g[pp]);
#pragma unroll
            for (int q = 0; q <= pp; ++q) am[tri(pp, q)] = fmaf(wj, J[q], am[tri(pp, q)]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < kNPk; ++i) am[i] = warp_sum(am[i]);
#pragma unroll
      for (int i = 0; i < kNP; ++i) g[i] = warp_sum(g[i]);
      __syncwarp();
      if (lane == 0) {  // every lane holds the totals
#pragma unroll
        for (int i = 0; i < kNPk; ++i) S.A[i] = am[i];
#pragma unroll
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
      }
      if (A.cov_out) {
        // parked for the batched covariance kernel, as in the filter path
        float* cv = A.cov_out + pix * 100;
        for (int j = lane; j < 100; j += 32)
          cv[j] = (status == VFISV_PIX_NAN_STATE || j >= kNPk) ? 0.0f : S.A[j];
      }
      __syncwarp();
      if (lane == 0) {
        map_retired(A, pix);
        S.pix = -1;
      }
      __syncwarp();
    }
  }
}

size_t wide_table_bytes(int nf, int nlam) { return (size_t)wide_table_floats(nf, nlam) * 4; }

static size_t wide_smem(int nf, int nlam, bool invert) {
  size_t b = (size_t)(wide_table_floats(nf, nlam) + kWWarps * wide_warp_floats(nf, invert)) * 4;
  if (invert) b += kWWarps * sizeof(WideWarpState);
  return ((b + 15) & ~(size_t)15) + 16;
}

bool wide_supported(int nf, int nlam) {
  return nf >= 1 && nf <= kWMaxF && nlam >= 1 && nlam <= kWMaxLam &&
         wide_smem(nf, nlam, true) <= 227 * 1024;
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
  nsm = sm_budget(nsm);
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
