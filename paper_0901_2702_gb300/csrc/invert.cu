// Persistent Levenberg-Marquardt kernel (Secs. 2 and 4): one pixel per
// thread slot, pixels drawn from a global work queue so that converged
// pixels retire and their slots refill.  Each iteration:
//   1. FP64 damped solve of the Jacobi-scaled normal equations (Eqs. 3-5),
//      Cholesky with a Jacobi-eigenvalue (SVD) fallback;
//   2. one fused FP32 pass over the wavelength grid giving the filtered
//      Stokes vector and the 6 per-wavelength Jacobian columns (Eqs. 8-9);
//   3. FP64 chi-square (Eq. 1) and the acceptance test (Fig. 6);
//   4. on success, J^T W J and J^T W r in compensated FP32 sums (Ogita-Rump-
//      Oishi Dot2), stored per slot in global scratch; damping by Table 2.
#include <math.h>

#include "common.cuh"
#include "dfloat.cuh"
#include "lm_device.cuh"
#include "solve.cuh"

namespace vfisv {

constexpr int kInvThreadsDefault = 128;  // pixel slots per CTA unless autotuned

// The same factorisation and solve in double-float arithmetic (the fast
// path of the damped step; FP64 is kept for the rare singular fallback).
__device__ __forceinline__ bool cholesky9_df(dfl (&L)[kNPk], dfl (&ri)[kNP]) {
#pragma unroll
  for (int j = 0; j < kNP; ++j) {
    dfl d = L[tri(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) d = df_fma(df_neg(L[tri(j, k)]), L[tri(j, k)], d);
    if (!(d.hi > 1e-10f)) return false;
    const dfl r = df_rsqrt(d);
    ri[j] = r;
    L[tri(j, j)] = df_mul(d, r);
#pragma unroll
    for (int i = j + 1; i < kNP; ++i) {
      dfl t = L[tri(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) t = df_fma(df_neg(L[tri(i, k)]), L[tri(j, k)], t);
      L[tri(i, j)] = df_mul(t, r);
    }
  }
  return true;
}

__device__ __forceinline__ void chol_solve9_df(const dfl (&L)[kNPk], const dfl (&ri)[kNP],
                                               dfl (&x)[kNP]) {
#pragma unroll
  for (int i = 0; i < kNP; ++i) {
    dfl t = x[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t = df_fma(df_neg(L[tri(i, k)]), x[k], t);
    x[i] = df_mul(t, ri[i]);
  }
#pragma unroll
  for (int i = kNP - 1; i >= 0; --i) {
    dfl t = x[i];
#pragma unroll
    for (int k = i + 1; k < kNP; ++k) t = df_fma(df_neg(L[tri(k, i)]), x[k], t);
    x[i] = df_mul(t, ri[i]);
  }
}

// The same step in double-float (the fast_solve option); the result is
// delta[i].hi + delta[i].lo.
__device__ __noinline__ void damped_step_df(const float* scr, int64_t ns, uint32_t free_mask, double eps,
                                         dfl (&delta)[kNP]) {
  dfl L[kNPk], sc[kNP], y[kNP];
  bool held[kNP];
  const dfl one_eps = df_add(df_from(1.0f), df_from_double(eps));
#pragma unroll
  for (int i = 0; i < kNP; ++i) {
    const float d = scr[(int64_t)tri(i, i) * ns];
    held[i] = !((free_mask >> i) & 1u) || !(d > 0.0f) || !isfinite(d);
    sc[i] = held[i] ? df_from(0.0f) : df_rsqrt(df_from(d));
    y[i] = held[i] ? df_from(0.0f) : df_mul(df_from(scr[(int64_t)(kNPk + i) * ns]), sc[i]);
  }
#pragma unroll
  for (int i = 0; i < kNP; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      dfl m;
      if (i == j)
        m = held[i] ? df_from(1.0f) : one_eps;
      else
        m = (held[i] || held[j])
                ? df_from(0.0f)
                : df_mul(df_mul(df_from(scr[(int64_t)tri(i, j) * ns]), sc[i]), sc[j]);
      L[tri(i, j)] = m;
    }
  dfl ri[kNP];
  if (!cholesky9_df(L, ri)) {
    // numerically singular: truncated eigen-decomposition in FP64
    double Ld[kNPk], scd[kNP], b[kNP], yd[kNP];
    bool h2[kNP];
    scaled_system(scr, ns, free_mask, eps, Ld, scd, h2);
#pragma unroll
    for (int i = 0; i < kNP; ++i) b[i] = df_to_double(y[i]);
    jacobi_pinv(Ld, b, yd, nullptr);
#pragma unroll
    for (int i = 0; i < kNP; ++i) y[i] = df_from_double(yd[i]);
  } else {
    chol_solve9_df(L, ri, y);
  }
#pragma unroll
  for (int i = 0; i < kNP; ++i) delta[i] = held[i] ? df_from(0.0f) : df_mul(sc[i], y[i]);
}

// Covariance (J^T W J)^+ at the final model, in parameter units, from the
// packed J^T W J at scr[e * ns].  Reads everything before writing `out`, so
// `out` may hold the packed matrix itself.  The Cholesky path runs in
// double-float (the fast_solve option); with try_only, returns false
// without writing when the factorisation fails (the caller then runs the
// FP64 eigen-decomposition path for that pixel).
__device__ __noinline__ bool covariance_df(const float* scr, int64_t ns, uint32_t free_mask,
                                           float* out, bool try_only) {
  uint32_t hmask = 0;
  dfl sc[kNP];
#pragma unroll
  for (int i = 0; i < kNP; ++i) {
    const float d = scr[(int64_t)tri(i, i) * ns];
    const bool h = !((free_mask >> i) & 1u) || !(d > 0.0f) || !isfinite(d);
    hmask |= (h ? 1u : 0u) << i;
    sc[i] = h ? df_from(0.0f) : df_rsqrt(df_from(d));
  }
  dfl L[kNPk], ri[kNP];
#pragma unroll
  for (int i = 0; i < kNP; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j)
      L[tri(i, j)] = (i == j) ? df_from(1.0f)
                     : (((hmask >> i) | (hmask >> j)) & 1u)
                         ? df_from(0.0f)
                         : df_mul(df_mul(df_from(scr[(int64_t)tri(i, j) * ns]), sc[i]), sc[j]);
  if (cholesky9_df(L, ri)) {
    // scr is no longer read.  In place: W = L^-1 (columns right to left,
    // each from the already inverted trailing block), then M^-1 = W^T W
    // (columns left to right) -- ~285 double-float FMAs instead of nine
    // solves (~810); then S M^-1 S, S = diag(sc), straight to out.
#pragma unroll
    for (int j = kNP - 1; j >= 0; --j) {
#pragma unroll
      for (int i = kNP - 1; i > j; --i) {
        dfl t = df_from(0.0f);
#pragma unroll
        for (int k = j + 1; k <= i; ++k) t = df_fma(L[tri(i, k)], L[tri(k, j)], t);
        L[tri(i, j)] = df_neg(df_mul(t, ri[j]));
      }
      L[tri(j, j)] = ri[j];
    }
#pragma unroll
    for (int j = 0; j < kNP; ++j)
#pragma unroll
      for (int i = j; i < kNP; ++i) {
        dfl t = df_from(0.0f);
#pragma unroll
        for (int k = i; k < kNP; ++k) t = df_fma(L[tri(k, i)], L[tri(k, j)], t);
        L[tri(i, j)] = t;
      }
#pragma unroll
    for (int j = 0; j < kNP; ++j)
#pragma unroll
      for (int i = j; i < kNP; ++i) {
        const float v = (((hmask >> i) | (hmask >> j)) & 1u)
                            ? 0.0f
                            : df_mul(df_mul(L[tri(i, j)], sc[i]), sc[j]).hi;
        out[i * 10 + j] = v;
        out[j * 10 + i] = v;
      }
    for (int k = 0; k < 10; ++k) {
      out[90 + k] = 0.0f;
      out[k * 10 + 9] = 0.0f;
    }
    return true;
  }
  if (try_only) return false;
  // numerically singular: truncated eigen-decomposition in FP64
  double Ld[kNPk], scd[kNP], Pd[kNPk];
  bool held[kNP];
  scaled_system(scr, ns, free_mask, 0.0, Ld, scd, held);
  jacobi_pinv(Ld, nullptr, nullptr, Pd);
  for (int i = 0; i < 10; ++i)
    for (int j = 0; j < 10; ++j) {
      float v = 0.0f;
      if (i < kNP && j < kNP && !held[i] && !held[j])
        v = (float)(scd[i] * scd[j] * ((i >= j) ? Pd[tri(i, j)] : Pd[tri(j, i)]));
      out[i * 10 + j] = v;
    }
  return true;
}

// ---- randomised restarts (Sec. 4.2) ----
// SplitMix64 (Steele, Lea & Flood 2014) read as a counter-based generator:
// output number `ctr` of the stream started at `seed` is the variant-13
// finaliser applied to seed + (ctr + 1) * golden-ratio increment.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Restart number k of pixel `pix`: uniform perturbations of the seven
// non-linear parameters with half-widths proportional to k (eta0 in its
// logarithm); S0, S1 and held parameters are left alone; bounds applied.
__device__ __forceinline__ void restart_model(float (&m)[10], long long pix, int k,
                                              uint64_t seed, uint32_t free_mask) {
  constexpr double amp[7] = {150.0, 10.0, 15.0, 0.25, 4.0, 0.05, 0.25};
#pragma unroll
  for (int p = 0; p < 7; ++p) {
    if (!((free_mask >> p) & 1u)) continue;
    const uint64_t z = splitmix64(seed, ((uint64_t)pix << 24) | ((uint64_t)k << 4) | (uint64_t)p);
    const double u = (double)(z >> 11) * 0x1.0p-53;  // [0, 1), 53 bits
    const double d = amp[p] * (double)k * (2.0 * u - 1.0);
    m[p] = (p == 3) ? (float)((double)m[p] * exp(d)) : (float)((double)m[p] + d);
  }
  apply_bounds(m);
}

__global__ void restart_perturb_kernel(const float* __restrict__ in, int64_t n, int64_t pix0,
                                       int k, uint32_t free_mask, uint64_t seed,
                                       float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float m[10];
#pragma unroll
    for (int j = 0; j < 10; ++j) m[j] = in[i * 10 + j];
    restart_model(m, pix0 + i, k, seed, free_mask);
#pragma unroll
    for (int j = 0; j < 10; ++j) out[i * 10 + j] = m[j];
  }
}

cudaError_t launch_restart_perturb(const float* in, int64_t n, int64_t pix0, int k,
                                   uint32_t free_mask, uint64_t seed, float* out, cudaStream_t s) {
  int64_t grid = (n + 255) / 256;
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  restart_perturb_kernel<<<(int)grid, 256, 0, s>>>(in, n, pix0, k, free_mask, seed, out);
  return cudaGetLastError();
}

// Weideman coefficients of this translation unit (set by invert_set_constants).
__constant__ Weideman c_W;

// Pool of dump buffers in shared memory: a buffer is [NACC][32] floats, one
// lane per column.  The filtered accumulators of a pass are needed only
// from the end of its wavelength loop to the end of the normal-equation
// build, a few per cent of an iteration, so a CTA keeps one buffer per
// four warps (at least one) and a warp (or the part of it that arrives
// together) takes one at the end of its loop.  The shared memory this
// frees goes to the L1 cache that holds the kernel's spilled registers.  owner[b] counts the lanes still using
// buffer b; each lane releases its own use, so divergence between the
// acquire and the release is harmless.  A holder waits on nothing, so the
// bounded wait below only covers the time other warps spend in their
// builds.
__host__ __device__ constexpr int dump_pool(int nt) { return nt >= 128 ? nt / 128 : 1; }

__device__ __forceinline__ int pool_acquire(int* owner, int npool, int* err) {
  const unsigned m = __activemask();
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  int b = -1;
  if (lane == leader) {
    const int users = __popc(m);
    const long long t0 = clock64();
    for (int it = 0; b < 0 && it < (1 << 24); ++it) {
      for (int i = 0; i < npool && b < 0; ++i)
        if (atomicCAS(&owner[i], 0, users) == 0) b = i;
      if (b < 0) {
        if (clock64() - t0 > (1ll << 31)) break;  // ~1 s at 2 GHz
        __nanosleep(32);
      }
    }
    if (b < 0) {  // reported; the pass goes on in a shared buffer (results invalid)
      atomicExch(err, kDevErrPoolWait);
      b = (threadIdx.x >> 5) % npool;
    }
  }
  b = __shfl_sync(m, b, leader);
  __threadfence_block();
  return b;
}

__device__ __forceinline__ void pool_release(int* owner, int b) {
  __threadfence_block();  // this lane's reads of the buffer come first
  atomicSub(&owner[b], 1);
}

// The fused pass over the wavelength grid, kept out of line so that its
// 168 accumulators get the whole register file; results go to the lane's
// column of a pooled dump buffer, whose index it returns.  With TPP > 1 the
// TPP consecutive lanes of a pixel each take every TPP-th grid point and
// then add their partial sums by xor-shuffles: every lane of the pixel ends
// with the same sums (IEEE addition is commutative, and the pairs are added
// in the same tree on every lane).
template <int NF, bool NM = false, int TPP = 1>
__device__ __noinline__ int fused_pass(const PixK P, const float* __restrict__ tab, int nlam,
                                       float* __restrict__ pool, int* owner, int npool,
                                       int* err) {
  constexpr int NACC = kRows * 4 * NF + (NM ? kNmRows * NF : 0);
  constexpr int S = ((NF + 1) + 3) & ~3;
  float acc[kRows][4][NF];
  float accn[NM ? kNmRows : 1][NF];
#pragma unroll
  for (int r = 0; r < kRows; ++r)
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int k = 0; k < NF; ++k) acc[r][s][k] = 0.0f;
#pragma unroll
  for (int r = 0; r < (NM ? kNmRows : 1); ++r)
#pragma unroll
    for (int k = 0; k < NF; ++k) accn[r][k] = 0.0f;
  const int nl = table_rows(tab, NF, nlam);
#pragma unroll 1
  for (int i = (TPP > 1) ? (int)(threadIdx.x % TPP) : 0; i < nl; i += TPP) {
    float T[NF];
    const float x = load_row<NF>(tab + (size_t)i * S, T);
    lambda_step<NF, true, NM>(c_W, P, x, T, acc, accn);
  }
  if constexpr (TPP > 1) {
    const int lane = threadIdx.x & 31;
    const unsigned pm = ((1u << TPP) - 1u) << (lane & ~(TPP - 1));
#pragma unroll
    for (int o = 1; o < TPP; o <<= 1)
#pragma unroll
      for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int k = 0; k < NF; ++k) acc[r][s][k] += __shfl_xor_sync(pm, acc[r][s][k], o);
  }
  const int b = pool_acquire(owner, npool, err);
  float* dump = pool + (size_t)b * NACC * 32 + (threadIdx.x & 31);
#pragma unroll
  for (int r = 0; r < kRows; ++r)
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int k = 0; k < NF; ++k) dump[((r * 4 + s) * NF + k) * 32] = acc[r][s][k];
  if constexpr (NM) {
    // the non-magnetic rows follow the magnetic ones
#pragma unroll
    for (int r = 0; r < kNmRows; ++r)
#pragma unroll
      for (int k = 0; k < NF; ++k) dump[(kRows * 4 * NF + r * NF + k) * 32] = accn[r][k];
  }
  return b;
}

// Per-slot LM state kept in shared memory (structure of arrays, one column
// per thread) so that the registers of the wavelength loop hold only its
// accumulators.
constexpr int kStateWords = 10 + 10 + 2 + 2 + 2 + 1 + 1;  // M, Mt, chi2b, eps, pix, it, near
// Layout: table | dump pool | state | pool owners (padded to 16 B) | work
// counters (4 x u64) | mbarrier.
constexpr int kNumCounters = 4;
__host__ __device__ constexpr size_t pool_owner_bytes(int nt) {
  return ((size_t)dump_pool(nt) * 4 + 15) & ~(size_t)15;
}
// nt threads per CTA serving nps pixel slots (nt / threads per pixel)
__host__ __device__ constexpr size_t invert_smem_bytes(int tabf, int nacc, int nt, int nps) {
  return (size_t)tabf * 4 + (size_t)dump_pool(nt) * nacc * 32 * 4 + (size_t)kStateWords * nps * 4 +
         pool_owner_bytes(nt) + 8 * kNumCounters + 16;
}

// RS: randomised restarts compiled in (A.restarts != 0).  DF: the damped
// solve in double-float and chi2 by a compensated FP32 sum (fast_solve);
// otherwise both in FP64.  AF: the filling factor alpha free (Sec. 2): the
// model mixes the magnetic and the non-magnetic (B = 0) profile, and the
// solve takes 10 parameters.  TPP: threads per pixel (1, 2 or 4): the lanes
// of a pixel split its wavelength points and otherwise run the same steps
// on the same data (every decision, and every value they write, is the
// same on each of them); a CTA of BS threads serves BS / TPP pixel slots.
template <int NF, int BS, bool RS, bool DF, bool AF = false, int TPP = 1>
__global__ void __launch_bounds__(BS, 1) invert_kernel(InvertArgs A) {
  static_assert(TPP == 1 || TPP == 2 || TPP == 4, "threads per pixel");
  static_assert(TPP == 1 || (!RS && !AF), "several threads per pixel: plain path only");
  constexpr int NOBS = 4 * NF;
  constexpr int NACC = kRows * 4 * NF + (AF ? kNmRows * NF : 0);
  constexpr int NP = AF ? 10 : kNP;        // parameters in the solve
  constexpr int NPK = NP * (NP + 1) / 2;   // packed J^T W J
  extern __shared__ __align__(16) float smem[];
  const int S = table_stride(NF);
  const int tabf = table_floats(NF, A.nlam);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nps = nt / TPP, ps = tid / TPP, q = tid % TPP;  // pixel slots, this slot, lane in it
  float* tab = smem;
  const int npool = dump_pool(nt);
  float* pool = smem + tabf;                      // [npool][NACC][32]
  float* sM = pool + (size_t)npool * NACC * 32;   // [10][nps] best model
  float* sMt = sM + 10 * nps;                     // [10][nps] trial model
  double* sChi = reinterpret_cast<double*>(sMt + 10 * nps);  // [nps]
  double* sEps = sChi + nps;                      // [nps]
  long long* sPix = reinterpret_cast<long long*>(sEps + nps);  // [nps]
  int* sIt = reinterpret_cast<int*>(sPix + nps);  // [nps]
  int* sNear = sIt + nps;  // [nps] last accepted step was close to the minimum (Hessian reuse)
  uint64_t* mbar =
      reinterpret_cast<uint64_t*>(smem + (invert_smem_bytes(tabf, NACC, nt, nps) - 16) / 4);
  // passes, accepted, retired, wavelength points evaluated
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(mbar) - kNumCounters;
  int* owner = reinterpret_cast<int*>(cnt) - pool_owner_bytes(nt) / 4;  // [npool]
  if (tid < npool) owner[tid] = 0;  // published by the barrier inside the table load
  if (tid < kNumCounters) cnt[tid] = 0;
  if (!tma_load_table(tab, A.table, (uint32_t)(tabf * sizeof(float)), mbar, A.err)) return;
  const float* tau = tab + (size_t)A.nlam * S;
  const int nrows = table_rows(tab, NF, A.nlam);
  const int64_t slot = (int64_t)blockIdx.x * nps + ps;
  const int64_t ns = A.nslots;
  float* scr = A.scratch + slot;
  const int dof = NOBS - A.nfree;
  const int64_t npix = A.npix_dev ? *A.npix_dev : A.npix;
#define ST(arr, j) arr[(j) * nps + ps]
  // restart state of this slot: best chi2, initial chi2; best J^T W J, J^T W r,
  // model; failed trials in a row, restart count, flags
  const RestartState R0(A.rs_state, ns);
  double* rsBest = R0.chi2 + slot;
  double* rsFirst = R0.chi2 + ns + slot;
  float* rsF = R0.f + slot;  // row j at rsF[j * ns]; model from row kScratchPerSlot
  int* rsFail = R0.i + slot;
  int* rsCount = R0.i + ns + slot;
  int* rsFlags = R0.i + 2 * ns + slot;
  constexpr int kEverConv = 1, kEverStall = 2, kPending = 4;

  sPix[ps] = -1;
  // lanes of one pixel (TPP > 1): they run the same steps on the same data,
  // but independent thread scheduling may let one run ahead of the other;
  // the slot's shared state is written only after both have read it (a
  // barrier of the pixel's lanes at the top of every iteration, and the
  // reads of the post-pass state taken into registers before a second one)
  const unsigned pm = (TPP > 1) ? (((1u << TPP) - 1u) << ((tid & 31) & ~(TPP - 1))) : 0u;
  while (true) {
    bool fresh = false, restart = false;
    if constexpr (TPP > 1) __syncwarp(pm);
    {
      long long pix = sPix[ps];
      if (pix < 0) {
        if (q == 0) pix = (long long)atomicAdd(A.queue, 1ull);
        if constexpr (TPP > 1) pix = __shfl_sync(pm, pix, (tid & 31) & ~(TPP - 1));
        if (pix >= npix) break;
        if (A.pix_list) pix = A.pix_list[pix];
        fresh = true;
        sPix[ps] = pix;
        const float* o = A.obs + pix * NOBS;
        const float* wv = weight_row(A, pix, NOBS);
        bool bad = false;
        float wsum = 0.0f, ic = -INFINITY;
#pragma unroll
        for (int j = 0; j < NOBS; ++j) {
          const float ov = o[j], ww = wv[j];
          bad |= !isfinite(ov) || !isfinite(ww);
          wsum += isfinite(ww) ? ww : 0.0f;
          if (j < NF) ic = fmaxf(ic, isfinite(ov) ? ov : 0.0f);
        }
        bad |= !(wsum > 0.0f);
        float Mt[10];
        if (A.init) {
          const float guess[10] = {500.f, 60.f, 45.f, 10.f, 35.f, 0.25f, 0.f, 0.25f, 0.75f, 1.f};
#pragma unroll
          for (int j = 0; j < 10; ++j) {
            const float v = A.init[pix * 10 + j];
            bad |= !isfinite(v);
            Mt[j] = isfinite(v) ? v : guess[j];
          }
        } else {
          Mt[0] = 500.f; Mt[1] = 60.f; Mt[2] = 45.f; Mt[3] = 10.f; Mt[4] = 35.f;
          Mt[5] = 0.25f; Mt[6] = 0.f;
          Mt[7] = 0.25f * ic;
          Mt[8] = 0.75f * ic / A.lk.mu;
        }
        if (!AF || !A.init) Mt[9] = 1.0f;
        apply_bounds(Mt);
        Mt[9] = fminf(fmaxf(Mt[9], 0.0f), 1.0f);
        if (bad) {
          for (int j = 0; j < 10; ++j) A.params_out[pix * 10 + j] = Mt[j];
          A.chi2_out[pix] = 0.0f;
          A.iters_out[pix] = 0;
          A.status_out[pix] = VFISV_PIX_BAD_INPUT;
          if (A.cov_out)
            for (int j = 0; j < 100; ++j) A.cov_out[pix * 100 + j] = 0.0f;
          if (q == 0) map_retired(A, pix);
          sPix[ps] = -1;
          continue;
        }
#pragma unroll
        for (int j = 0; j < 10; ++j) ST(sMt, j) = Mt[j];
        sIt[ps] = 0;
        sEps[ps] = A.eps0;
        sNear[ps] = 0;
        if (RS) {
          *rsBest = INFINITY;
          *rsFail = 0;
          *rsCount = 0;
          *rsFlags = 0;
        }
      } else if (RS && (*rsFlags & kPending)) {
        // restart pass: the best model so far, perturbed
        const int k = ++*rsCount;
        float Mt[10];
#pragma unroll
        for (int j = 0; j < 10; ++j) Mt[j] = rsF[(kScratchPerSlot + j) * ns];
        restart_model(Mt, pix, k, A.seed, A.free_mask);
#pragma unroll
        for (int j = 0; j < 10; ++j) ST(sMt, j) = Mt[j];
        restart = true;
      } else {
        float Mt[10];
        if constexpr (DF) {
          dfl d[kNP];
          damped_step_df(scr, ns, A.free_mask, sEps[ps], d);
#pragma unroll
          for (int j = 0; j < kNP; ++j) {
            const dfl t = two_sum(ST(sM, j), d[j].hi);
            Mt[j] = t.hi + (t.lo + d[j].lo);  // the FP32 model nearest M + delta
          }
        } else {
          double d[NP];
          damped_step_fp64<NP>(scr, ns, A.free_mask, sEps[ps], d);
#pragma unroll
          for (int j = 0; j < NP; ++j) Mt[j] = (float)((double)ST(sM, j) + d[j]);
        }
        if constexpr (AF)
          Mt[9] = fminf(fmaxf(Mt[9], 0.0f), 1.0f);
        else
          Mt[9] = 1.0f;
        apply_bounds(Mt);
#pragma unroll
        for (int j = 0; j < 10; ++j) ST(sMt, j) = Mt[j];
      }
    }

    // ---- fused synthesis + Jacobian at the trial model (Secs. 3 and 4.4) ----
    const int dbuf = fused_pass<NF, AF, TPP>(make_pixk(A.lk, ST(sMt, 0), ST(sMt, 1), ST(sMt, 3),
                                                  ST(sMt, 4), ST(sMt, 5), ST(sMt, 6)),
                                        tab, A.nlam, pool, owner, npool, A.err);
    const float* dump = pool + (size_t)dbuf * NACC * 32 + (tid & 31);
    auto D = [&](int r, int s, int k) { return dump[((r * 4 + s) * NF + k) * 32]; };
    // non-magnetic Stokes I rows (AF): value, then the E, D, A, V rows
    auto N = [&](int r, int k) { return dump[(kRows * 4 * NF + r * NF + k) * 32]; };
    const float alf = AF ? ST(sMt, 9) : 1.0f;

    const long long pix = sPix[ps];
    const float* o = A.obs + pix * NOBS;
    const float* wv = weight_row(A, pix, NOBS);
    // the slot state this iteration updates, read before any lane writes it
    const int it_in = sIt[ps];
    const double chi2_in = sChi[ps], eps_in = sEps[ps];
    const int near_in = sNear[ps];
    if constexpr (TPP > 1) __syncwarp(pm);

    // ---- model, residual and chi-square (Eq. 1, FP64) ----
    float c2p, s2p;
    sincosf(2.0f * ST(sMt, 2) * kDeg, &s2p, &c2p);
    const float mus1 = A.lk.mu * ST(sMt, 8);
    const float s0 = ST(sMt, 7);
    float syn[NOBS];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      // with alpha free: alpha x magnetic + (1 - alpha) x non-magnetic
      const float q0 = alf * D(0, 1, k), u0 = alf * D(0, 2, k);
      const float yI = AF ? fmaf(alf, D(0, 0, k) - N(0, k), N(0, k)) : D(0, 0, k);
      syn[k] = fmaf(s0, tau[k], mus1 * yI);
      syn[NF + k] = mus1 * fmaf(c2p, q0, -s2p * u0);
      syn[2 * NF + k] = mus1 * fmaf(s2p, q0, c2p * u0);
      syn[3 * NF + k] = mus1 * (alf * D(0, 3, k));
    }
    double c2;
    if constexpr (DF) {
      // compensated FP32 sum of w r^2 (the residuals themselves carry the
      // FP32 synthesis error, ~1e-4 of chi2)
      Dot2 q{0.0f, 0.0f};
#pragma unroll
      for (int j = 0; j < NOBS; ++j) {
        const float r = o[j] - syn[j];
        q.add(wv[j] * r, r);
      }
      c2 = ((double)q.s + (double)q.c) / (double)dof;
    } else {
      c2 = 0.0;
#pragma unroll
      for (int j = 0; j < NOBS; ++j) {
        const double r = (double)(o[j] - syn[j]);
        c2 = fma((double)wv[j] * r, r, c2);
      }
      c2 /= (double)dof;
    }

    if (A.counters && q == 0) {
      atomicAdd(&cnt[0], 1ull);
      atomicAdd(&cnt[3], (unsigned long long)nrows);
    }
    bool accept, retire = false;
    int status = VFISV_PIX_MAXITER;
    int it = it_in;
    double rel_acc = INFINITY;  // relative chi2 decrease of an accepted trial step
    if (fresh) {
      accept = isfinite(c2);
      if (!accept) {
        retire = true;
        status = VFISV_PIX_NAN_STATE;
      }
      if (RS) *rsFirst = c2;
    } else if (RS && restart) {
      // a new segment starts at the perturbed model whatever its chi2; a
      // non-finite one leaves the restart pending (retried with k + 1)
      ++it;
      accept = isfinite(c2);
      if (accept) {
        sEps[ps] = A.eps0;
        *rsFail = 0;
        *rsFlags &= ~kPending;
      }
    } else {
      ++it;
      const double chi2b = chi2_in;
      accept = isfinite(c2) && c2 < chi2b;
      const double eps_used = eps_in;
      const double eps = eps_update(eps_used, accept);
      sEps[ps] = eps;
      bool conv = false, stall = false;
      if (accept) {
        const double rel = (chi2b - c2) / chi2b;
        rel_acc = rel;
        conv = rel < A.conv_rtol && eps_used <= A.conv_eps;
      } else {
        stall = eps >= 1e12;
      }
      if (!RS) {
        if (conv || stall) {
          retire = true;
          status = conv ? VFISV_PIX_CONVERGED : VFISV_PIX_STALLED;
        }
      } else {
        int fl = *rsFlags;
        const int nfail = accept ? 0 : *rsFail + 1;
        *rsFail = nfail;
        fl |= (conv ? kEverConv : 0) | (stall ? kEverStall : 0);
        bool trig = false;
        if (conv || stall) {
          if (A.restarts & kRestartAtConvergence) trig = true;
          else retire = true;
        }
        // (a) at iteration 10, chi2 not down by a decade from its first value
        // (the best chi2 so far counts, including this trial's)
        if ((A.restarts & kRestartA) && it == 10) {
          const double best = (accept && c2 < *rsBest) ? c2 : *rsBest;
          trig |= !(best <= *rsFirst / 10.0);
        }
        if ((A.restarts & kRestartB) && nfail >= 5) trig = true;  // (b)
        if (trig && !retire) fl |= kPending;
        *rsFlags = fl;
      }
    }
    sIt[ps] = it;
    if (A.counters && q == 0 && accept && !fresh) atomicAdd(&cnt[1], 1ull);

    if (accept) {
      // ---- J^T W J and J^T W r at the new best model (compensated FP32) ----
#pragma unroll
      for (int j = 0; j < 10; ++j) ST(sM, j) = ST(sMt, j);
      sChi[ps] = c2;
      // Hessian reuse (Sec. 4.4): this and the previous accepted step both
      // close to the minimum -> keep J^T W J, rebuild J^T W r only
      const bool near = rel_acc < A.hess_reuse;
      const bool keepA = near && near_in;
      sNear[ps] = near;
      // rows from the lane's column of the dump buffer (shared memory)
      struct {
        const float* dump;
        const float* o;
        const float* wv;
        ObsRead<NF> ov;
        __device__ void issue(int k, int s) { ov.issue(o, wv, k, s); }
        __device__ void take(int k, int s, ObsRows& rw) {
          rw.obs = ov.o;
          rw.w = ov.w;
          const int sa = obs_sa(s), sb = obs_sb(s);
#pragma unroll
          for (int r = 0; r < kRows; ++r) {
            rw.a[r] = dump[((r * 4 + sa) * NF + k) * 32];
            rw.b[r] = dump[((r * 4 + sb) * NF + k) * 32];
          }
          if constexpr (AF)
#pragma unroll
            for (int r = 0; r < kNmRows; ++r) rw.n[r] = dump[(kRows * 4 * NF + r * NF + k) * 32];
        }
      } fetch{dump, o, wv, {}};
      build_normal_equations<NF, NP, AF, false>(fetch, tau, scr, ns, mus1, c2p, s2p, s0,
                                                alf, A.lk.mu,
                                                row_scale(A.lk, ST(sMt, 3), ST(sMt, 4)), keepA,
                                                true);
      if (RS && c2 < *rsBest) {
        // a new best over all segments: keep it with its normal equations
        *rsBest = c2;
#pragma unroll 1
        for (int i = 0; i < kScratchPerSlot; ++i) rsF[i * ns] = scr[(int64_t)i * ns];
#pragma unroll
        for (int j = 0; j < 10; ++j) rsF[(kScratchPerSlot + j) * ns] = ST(sM, j);
      }
    }
    pool_release(owner, dbuf);  // the filtered rows are not read past this point
    if (!retire && it >= A.max_iter) retire = true;  // status stays MAXITER

    if (retire) {
      double chi2b = accept ? c2 : chi2_in;
      // with restarts the result is the best model of all segments
      const float* src = scr;
      if (status == VFISV_PIX_NAN_STATE) {
#pragma unroll
        for (int j = 0; j < 10; ++j) ST(sM, j) = ST(sMt, j);
        chi2b = c2;
      } else if (RS) {
        const int fl = *rsFlags;
        status = (fl & kEverConv) ? VFISV_PIX_CONVERGED
                                  : ((fl & kEverStall) ? VFISV_PIX_STALLED : VFISV_PIX_MAXITER);
        chi2b = *rsBest;
#pragma unroll
        for (int j = 0; j < 10; ++j) ST(sM, j) = rsF[(kScratchPerSlot + j) * ns];
        src = rsF;
      }
      for (int j = 0; j < 10; ++j) A.params_out[pix * 10 + j] = ST(sM, j);
      A.chi2_out[pix] = (float)chi2b;
      A.iters_out[pix] = it;
      A.status_out[pix] = status;
      if (A.cov_out) {
        // the covariance itself is computed by covariance_kernel for all
        // pixels at once (full warps); here the pixel's J^T W J is parked in
        // its own output row
        float* cv = A.cov_out + pix * 100;
        if (status == VFISV_PIX_NAN_STATE) {
          for (int j = 0; j < 100; ++j) cv[j] = 0.0f;
        } else {
          // all 45 loads first (one retiring lane runs this while its warp
          // waits), then 400-byte-aligned vector stores into the row
          constexpr int NPK4 = (NPK + 3) & ~3;
          float v[NPK4];
#pragma unroll
          for (int j = 0; j < NPK4; ++j) v[j] = (j < NPK) ? src[(int64_t)j * ns] : 0.0f;
          if ((reinterpret_cast<uintptr_t>(A.cov_out) & 15u) == 0) {  // rows are 400 B
            float4* c4 = reinterpret_cast<float4*>(cv);
#pragma unroll
            for (int j = 0; j < NPK4 / 4; ++j)
              c4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < NPK; ++j) cv[j] = v[j];
          }
        }
      }
      if (q == 0) map_retired(A, pix);
      sPix[ps] = -1;
      if (A.counters && q == 0) atomicAdd(&cnt[2], 1ull);
    }
  }
#undef ST
  if (A.counters) {
    __syncthreads();  // every slot of the CTA has left the queue loop
    if (tid < kNumCounters) atomicAdd(A.counters + tid, cnt[tid]);
  }
}

// Covariance of every pixel that finished with a model, from the packed
// J^T W J parked in the pixel's output row.  Cholesky runs one pixel per
// thread; the rare pixels whose matrix is numerically singular go to a
// shared-memory queue and are drained by consecutive threads, so the costly
// eigen-decomposition runs in (nearly) full warps instead of stalling every
// warp that happens to hold one such pixel.
constexpr int kCovThreads = 128;
constexpr int kCovQueue = 2 * kCovThreads;
template <bool DF, int NPAR = kNP>
__global__ void __launch_bounds__(kCovThreads) covariance_kernel(float* cov,
                                                                 const int32_t* status,
                                                                 int64_t npix_max,
                                                                 const int64_t* npix_dev,
                                                                 uint32_t free_mask) {
  __shared__ int64_t queue[kCovQueue];
  __shared__ int qn;
  const int64_t npix = npix_dev ? *npix_dev : npix_max;
  if (threadIdx.x == 0) qn = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // every thread of the block runs the same number of rounds
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < npix; base += stride) {
    const int64_t p = base + threadIdx.x;
    if (p < npix) {
      const int st = status[p];
      if (st == VFISV_PIX_CONVERGED || st == VFISV_PIX_MAXITER || st == VFISV_PIX_STALLED) {
        const bool ok = DF ? covariance_df(cov + p * 100, 1, free_mask, cov + p * 100, true)
                           : covariance_fp64<NPAR>(cov + p * 100, 1, free_mask, cov + p * 100,
                                                   true);
        if (!ok) {
          const int slot = atomicAdd(&qn, 1);
          queue[slot] = p;  // slot < kCovQueue: drained below before it can fill
        }
      }
    }
    __syncthreads();
    const bool last = base + stride >= npix;
    if (qn >= kCovThreads || last) {
      const int n = qn;
      for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (DF)
          covariance_df(cov + queue[i] * 100, 1, free_mask, cov + queue[i] * 100, false);
        else
          covariance_fp64<NPAR>(cov + queue[i] * 100, 1, free_mask, cov + queue[i] * 100, false);
      __syncthreads();
      if (threadIdx.x == 0) qn = 0;
    }
    __syncthreads();
  }
}

cudaError_t launch_covariance(float* cov, const int32_t* status, int64_t npix,
                              const int64_t* npix_dev, uint32_t free_mask, int fast_solve,
                              cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  nsm = sm_budget(nsm);
  // a few blocks per SM, each sweeping many pixels so its fallback queue fills
  int64_t grid = (npix + kCovThreads - 1) / kCovThreads;
  if (grid > (int64_t)nsm * 4) grid = (int64_t)nsm * 4;
  if (grid < 1) grid = 1;
  if (fast_solve)
    covariance_kernel<true><<<(int)grid, kCovThreads, 0, s>>>(cov, status, npix, npix_dev, free_mask);
  else if (free_mask & (1u << 9))  // the filling factor free: 10 parameters
    covariance_kernel<false, 10><<<(int)grid, kCovThreads, 0, s>>>(cov, status, npix, npix_dev,
                                                                    free_mask);
  else
    covariance_kernel<false><<<(int)grid, kCovThreads, 0, s>>>(cov, status, npix, npix_dev, free_mask);
  return cudaGetLastError();
}

template <int BS, bool RS, bool DF, bool AF = false, int TPP = 1>
static cudaError_t slots_for(int nlam, int64_t npix, int64_t* nslots, int* grid, size_t* smem) {
  auto kern = invert_kernel<6, BS, RS, DF, AF, TPP>;
  constexpr int NPS = BS / TPP;  // pixel slots per CTA
  const size_t sm =
      invert_smem_bytes(table_floats(6, nlam), kRows * 4 * 6 + (AF ? kNmRows * 6 : 0), BS, NPS);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  nsm = sm_budget(nsm);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, BS, sm);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorLaunchOutOfResources;
  int64_t g = (int64_t)nsm * per;
  const int64_t need = (npix + NPS - 1) / NPS;
  if (need < g) g = need;
  if (g < 1) g = 1;
  *grid = (int)g;
  *smem = sm;
  *nslots = g * NPS;
  return cudaSuccess;
}

template <bool DF, int TPP>
static cudaError_t slots_bs(int bs, int nlam, int64_t npix, int64_t* nslots, int* grid,
                            size_t* smem) {
  switch (bs) {
    case 64: return slots_for<64, false, DF, false, TPP>(nlam, npix, nslots, grid, smem);
    case 256: return slots_for<256, false, DF, false, TPP>(nlam, npix, nslots, grid, smem);
    default: return slots_for<128, false, DF, false, TPP>(nlam, npix, nslots, grid, smem);
  }
}

template <bool DF>
static cudaError_t invert_slots_t(int nlam, int64_t npix, int restarts, int64_t* nslots,
                                  int* grid, int* block, int* tpp, size_t* smem) {
  if (restarts) {  // compiled for the default slot count only
    *block = kInvThreadsDefault;
    *tpp = 1;
    return slots_for<kInvThreadsDefault, true, DF>(nlam, npix, nslots, grid, smem);
  }
  const int bs = (*block == 64 || *block == 256) ? *block : kInvThreadsDefault;
  const int t = (*tpp == 2 || *tpp == 4) ? *tpp : 1;
  *block = bs;
  *tpp = t;
  switch (t) {
    case 2: return slots_bs<DF, 2>(bs, nlam, npix, nslots, grid, smem);
    case 4: return slots_bs<DF, 4>(bs, nlam, npix, nslots, grid, smem);
    default: return slots_bs<DF, 1>(bs, nlam, npix, nslots, grid, smem);
  }
}

cudaError_t invert_slots(int nf, int nlam, int64_t npix, int restarts, int fast_solve,
                         int alpha_free, int64_t* nslots, int* grid, int* block, int* tpp,
                         size_t* smem) {
  if (nf != 6) return cudaErrorInvalidValue;
  if (alpha_free) {  // compiled for the default slot count, FP64 solve, no restarts
    if (restarts || fast_solve) return cudaErrorInvalidValue;
    *block = kInvThreadsDefault;
    *tpp = 1;
    return slots_for<kInvThreadsDefault, false, false, true>(nlam, npix, nslots, grid, smem);
  }
  if (*block == kInvWsBlock) {
    if (!restarts && !fast_solve) {  // the warp-specialised kernel
      *tpp = 1;
      return invert_ws_slots(nlam, npix, nslots, grid, smem);
    }
    *block = kInvThreadsDefault;  // not compiled for this configuration
  }
  return fast_solve ? invert_slots_t<true>(nlam, npix, restarts, nslots, grid, block, tpp, smem)
                    : invert_slots_t<false>(nlam, npix, restarts, nslots, grid, block, tpp, smem);
}

cudaError_t invert_set_constants(const Weideman& W) {
  const cudaError_t e = cudaMemcpyToSymbol(c_W, &W, sizeof(W));
  return e != cudaSuccess ? e : invert_ws_set_constants(W);
}

template <bool DF, int TPP>
static cudaError_t launch_bs(const InvertArgs& a, int grid, int block, size_t smem,
                             cudaStream_t s) {
  switch (block) {
    case 64: invert_kernel<6, 64, false, DF, false, TPP><<<grid, 64, smem, s>>>(a); break;
    case 256: invert_kernel<6, 256, false, DF, false, TPP><<<grid, 256, smem, s>>>(a); break;
    case 128: invert_kernel<6, 128, false, DF, false, TPP><<<grid, 128, smem, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <bool DF>
static cudaError_t launch_invert_t(const InvertArgs& a, int grid, int block, int tpp,
                                   size_t smem, cudaStream_t s) {
  if (a.restarts) {
    if (block != kInvThreadsDefault || tpp != 1 || !a.rs_state) return cudaErrorInvalidValue;
    invert_kernel<6, kInvThreadsDefault, true, DF><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
  }
  switch (tpp) {
    case 1: return launch_bs<DF, 1>(a, grid, block, smem, s);
    case 2: return launch_bs<DF, 2>(a, grid, block, smem, s);
    case 4: return launch_bs<DF, 4>(a, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_invert(const InvertArgs& a, int nf, int grid, int block, int tpp, size_t smem,
                          cudaStream_t s) {
  if (nf != 6) return cudaErrorInvalidValue;
  if (a.free_mask & (1u << 9)) {
    if (a.restarts || a.fast_solve || block != kInvThreadsDefault || tpp != 1)
      return cudaErrorInvalidValue;
    invert_kernel<6, kInvThreadsDefault, false, false, true><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
  }
  if (block == kInvWsBlock) {
    if (a.restarts || a.fast_solve || tpp != 1) return cudaErrorInvalidValue;
    return launch_invert_ws(a, grid, smem, s);
  }
  return a.fast_solve ? launch_invert_t<true>(a, grid, block, tpp, smem, s)
                      : launch_invert_t<false>(a, grid, block, tpp, smem, s);
}

}  // namespace vfisv
