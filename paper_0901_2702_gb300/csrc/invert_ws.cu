// Warp-specialised persistent Levenberg-Marquardt kernel (Secs. 2 and 4)
// for the default configuration: 6 filter positions, FP64 damped solve and
// chi2, filling factor held, no restarts, one pixel per slot.  Same
// iteration, same arithmetic and same results as invert_kernel; only the
// division of the work between warps differs.
//
// One CTA per SM, 384 threads in three warpgroups.  Warpgroup 0 (one warp
// per SM sub-partition) only runs the fused FP32 synthesis + Jacobian +
// filter pass over the wavelength grid (Secs. 3, 4.4).  Warpgroups 1 and 2
// own the pixel slots, one per thread, and run everything else: the FP64
// chi2 and the acceptance test (Eq. 1, Fig. 6), the compensated J^T W J
// build (Eqs. 3-4), the FP64 damped solve (Eqs. 4-5), retirement and the
// work queue.  Producer warp p serves consumer warps 4 + p and 8 + p (its
// batches 0 and 1, 32 slots each) in turn: while it synthesises one batch's
// trial models, the other batch's consumer warp works through its last
// pass, so the FP32 pipe, the FP64 pipe and the latency of the solve
// overlap in every sub-partition.
//
// The 168 filtered rows of a pass go from producer to consumer through
// tensor memory: producer lane l of warp p writes TMEM lane 32p + l, in the
// batch's column range; consumer warps 4 + p and 8 + p sit in the same
// sub-partition (warp id mod 4) and read the same lanes.  Within a batch's
// range, the seven rows of Stokes s of filter k fill the 8-column group
// k * 4 + s (row r at column r), and the unit-S1 Stokes values of all
// observables follow contiguously for the chi2.  The slots' LM state
// (models, normal equations, damping, best chi2, iteration, flags) lives in
// shared memory.  Hand-offs are mbarriers with bounded waits: full[b] (rows
// of batch b written), empty[b] (rows read and the next trial models of
// batch b written).  Registers: the
// producers raise their limit to 232 (the pass's accumulators without
// spills), the consumers drop to 136 (setmaxnreg): three warps per
// sub-partition against two for invert_kernel.
#include <math.h>

#include "common.cuh"
#include "lm_device.cuh"
#include "solve.cuh"

namespace vfisv {

// Weideman coefficients of this translation unit (set by invert_set_constants).
__constant__ Weideman c_Wws;

namespace {

constexpr int kWsWarps = 12;
constexpr int kWsThreadsN = kWsWarps * 32;
constexpr int kWsBatches = 8;                  // consumer warps
constexpr int kWsSlotsN = kWsBatches * 32;     // pixel slots per CTA
constexpr int kWsProdRegs = 232, kWsConsRegs = 136;
constexpr int kWsTmemCols = 512;
constexpr int kWsGroup = 8;                    // columns per (filter, Stokes) group
constexpr int kWsBatchCols = 256;              // batch 1 of a producer starts here
constexpr int kFlagNear = 1, kFlagFresh = 2;
static_assert(kWsWarps == 4 + kWsBatches, "one producer warp per sub-partition");
static_assert(kWsBatches == 8, "each producer warp serves two consumer warps");
// a batch's 7-row groups and its row-0 copy fit its column range, and both
// batches fit the allocation (a power of two, at most 512 columns)
static_assert(4 * 6 * kWsGroup + 4 * 6 <= kWsBatchCols, "batch columns");
static_assert(kWsBatchCols + 4 * 6 * kWsGroup + 4 * 6 <= kWsTmemCols && kWsTmemCols <= 512,
              "tensor-memory columns");
static_assert(kWsProdRegs % 8 == 0 && kWsConsRegs % 8 == 0, "setmaxnreg counts");

// Shared-memory layout: the filter table, then these arrays (byte offsets
// from the start of shared memory), structure of arrays over the slots.
struct WsSmem {
  size_t mt, m, scr, pix, eps, chi2, it, flags, fin, cnt, tslot, bars, tbar, total;
  __host__ __device__ explicit WsSmem(int tabf) {
    size_t o = (size_t)tabf * 4;
    mt = o;   o += (size_t)10 * kWsSlotsN * 4;          // trial models [10][slots]
    m = o;    o += (size_t)10 * kWsSlotsN * 4;          // best models [10][slots]
    scr = o;  o += (size_t)(kNPk + kNP) * kWsSlotsN * 4;  // normal equations [54][slots]
    pix = o;  o += (size_t)kWsSlotsN * 8;               // pixel of each slot (-1: idle)
    eps = o;  o += (size_t)kWsSlotsN * 8;               // damping
    chi2 = o; o += (size_t)kWsSlotsN * 8;               // chi2 of the best model
    it = o;   o += (size_t)kWsSlotsN * 4;               // iterations
    flags = o; o += (size_t)kWsSlotsN * 4;              // kFlagNear | kFlagFresh
    fin = o;  o += 16 * 4;                               // batch finished flags
    cnt = o;  o += 4 * 8;                                // work counters
    tslot = o; o += 16;                                  // tensor-memory base address
    bars = o; o += 2 * kWsBatches * 8;                   // full[8], empty[8]
    tbar = o; o += 16;                                   // table copy
    total = o;
  }
};

__device__ __forceinline__ void ws_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool ws_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the phase of parity `parity`; false after ~1 s.  Called by whole
// warps, and the answer is the warp's: a lane that reaches the limit just as
// another sees the phase complete must not split the warp ahead of the
// warp-wide tensor-memory instructions that follow.
__device__ __forceinline__ bool ws_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  bool ok = false;
  for (int it = 0; it < (1 << 26) && !ok; ++it) {
    ok = ws_try(bar, parity);
    if (!ok && clock64() - t0 > (1ll << 31)) break;
  }
  return __all_sync(0xffffffffu, ok) != 0;
}

__device__ __forceinline__ void tc_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Eight FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tm_st8(uint32_t taddr, float v0, float v1, float v2, float v3,
                                       float v4, float v5, float v6, float v7) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
      "r"(__float_as_uint(v0)), "r"(__float_as_uint(v1)), "r"(__float_as_uint(v2)),
      "r"(__float_as_uint(v3)), "r"(__float_as_uint(v4)), "r"(__float_as_uint(v5)),
      "r"(__float_as_uint(v6)), "r"(__float_as_uint(v7))
      : "memory");
}

__device__ __forceinline__ void tm_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}

// Completes the loads issued before it; the registers are tied to the wait
// so that no use of them is scheduled ahead of it.
__device__ __forceinline__ void tm_wait16(uint32_t (&a)[8], uint32_t (&b)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]),
                 "+r"(a[6]), "+r"(a[7]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]),
                 "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7])::"memory");
}

__device__ __forceinline__ void tm_wait24(uint32_t (&a)[8], uint32_t (&b)[8], uint32_t (&c)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]),
                 "+r"(a[6]), "+r"(a[7]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]),
                 "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]), "+r"(c[0]), "+r"(c[1]),
                 "+r"(c[2]), "+r"(c[3]), "+r"(c[4]), "+r"(c[5]), "+r"(c[6]), "+r"(c[7])::"memory");
}

template <int NF>
__device__ __forceinline__ bool ws_producer(const InvertArgs& A, int p, uint32_t tlane,
                                            const float* __restrict__ tab, int nrows,
                                            const float* sMt, const long long* sPix,
                                            const int* fin, uint32_t bar_full,
                                            uint32_t bar_empty) {
  constexpr int S = ((NF + 1) + 3) & ~3;
  constexpr int NOBS = 4 * NF;
  const int lane = threadIdx.x & 31;
  uint32_t pe = 0u, done = 0u;  // bit x: parity of batch x's empty barrier; batch x finished
  while (done != 3u) {
#pragma unroll 1
    for (int x = 0; x < 2; ++x) {
      if ((done >> x) & 1u) continue;
      const int b = p + 4 * x;
      if (!ws_wait(bar_empty + 8 * b, (pe >> x) & 1u)) return false;
      pe ^= 1u << x;
      __syncwarp();
      tc_after();
      if (*(volatile const int*)(fin + b)) {
        done |= 1u << x;
        continue;
      }
      const int slot = b * 32 + lane;
      float acc[kRows][4][NF];
#pragma unroll
      for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int k = 0; k < NF; ++k) acc[r][s][k] = 0.0f;
      if (sPix[slot] >= 0) {
        const PixK P = make_pixk(A.lk, sMt[0 * kWsSlotsN + slot], sMt[1 * kWsSlotsN + slot],
                                 sMt[3 * kWsSlotsN + slot], sMt[4 * kWsSlotsN + slot],
                                 sMt[5 * kWsSlotsN + slot], sMt[6 * kWsSlotsN + slot]);
#pragma unroll 1
        for (int i = 0; i < nrows; ++i) {
          float T[NF];
          const float xw = load_row<NF>(tab + (size_t)i * S, T);
          lambda_step<NF, true>(c_Wws, P, xw, T, acc);
        }
      }
      // every lane of the warp stores (the tensor-memory stores are
      // warp-wide); idle slots store zeros
      __syncwarp();
      const uint32_t tb = tlane + (x ? (uint32_t)kWsBatchCols : 0u);
#pragma unroll
      for (int k = 0; k < NF; ++k)
#pragma unroll
        for (int s = 0; s < 4; ++s)
          tm_st8(tb + (uint32_t)((k * 4 + s) * kWsGroup), acc[0][s][k], acc[1][s][k],
                 acc[2][s][k], acc[3][s][k], acc[4][s][k], acc[5][s][k], acc[6][s][k], 0.0f);
#pragma unroll
      for (int j = 0; j < NOBS; j += 8)
        tm_st8(tb + (uint32_t)(4 * NF * kWsGroup + j), acc[0][j / NF][j % NF],
               acc[0][(j + 1) / NF][(j + 1) % NF], acc[0][(j + 2) / NF][(j + 2) % NF],
               acc[0][(j + 3) / NF][(j + 3) % NF], acc[0][(j + 4) / NF][(j + 4) % NF],
               acc[0][(j + 5) / NF][(j + 5) % NF], acc[0][(j + 6) / NF][(j + 6) % NF],
               acc[0][(j + 7) / NF][(j + 7) % NF]);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      tc_before();
      __syncwarp();
      ws_arrive(bar_full + 8 * b);
    }
  }
  return true;
}

template <int NF>
__device__ __forceinline__ bool ws_consumer(const InvertArgs& A, int b, uint32_t tc,
                                            const float* __restrict__ tab, int nrows,
                                            float* sMt, float* sM, float* sScr, long long* sPix,
                                            double* sEps, double* sChi, int* sIt, int* sFlags,
                                            int* fin, unsigned long long* cnt, uint32_t bar_full,
                                            uint32_t bar_empty) {
  constexpr int NOBS = 4 * NF;
  constexpr int NP = kNP, NPK = kNPk;
  constexpr int64_t ns = kWsSlotsN;
  static_assert(NF == 6, "the tensor-memory layout holds 6 filter positions");
  const int lane = threadIdx.x & 31;
  const int slot = b * 32 + lane;
  float* Mt = sMt + slot;
  float* M = sM + slot;
  float* scr = sScr + slot;
  const float* tau = tab + (size_t)A.nlam * table_stride(NF);
  const int dof = NOBS - A.nfree;
  const int64_t npix = A.npix_dev ? *A.npix_dev : A.npix;
  // the slot's LM state stays in shared memory between passes (fewer live
  // registers beside the FP64 solve)
  long long pix = -1;

  // the next pixel of the queue into this slot: its starting model as the
  // trial model (bad inputs are answered on the spot); -1 when none is left
  auto next_pixel = [&]() {
    for (;;) {
      const unsigned long long q = atomicAdd(A.queue, 1ull);
      if ((long long)q >= npix) {
        pix = -1;
        return;
      }
      const long long pq = A.pix_list ? A.pix_list[q] : (long long)q;
      const float* o = A.obs + pq * NOBS;
      const float* wv = weight_row(A, pq, NOBS);
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
      float m[10];
      if (A.init) {
        const float guess[10] = {500.f, 60.f, 45.f, 10.f, 35.f, 0.25f, 0.f, 0.25f, 0.75f, 1.f};
#pragma unroll
        for (int j = 0; j < 10; ++j) {
          const float v = A.init[pq * 10 + j];
          bad |= !isfinite(v);
          m[j] = isfinite(v) ? v : guess[j];
        }
      } else {
        m[0] = 500.f; m[1] = 60.f; m[2] = 45.f; m[3] = 10.f; m[4] = 35.f;
        m[5] = 0.25f; m[6] = 0.f;
        m[7] = 0.25f * ic;
        m[8] = 0.75f * ic / A.lk.mu;
      }
      m[9] = 1.0f;
      apply_bounds(m);
      if (bad) {
        for (int j = 0; j < 10; ++j) A.params_out[pq * 10 + j] = m[j];
        A.chi2_out[pq] = 0.0f;
        A.iters_out[pq] = 0;
        A.status_out[pq] = VFISV_PIX_BAD_INPUT;
        if (A.cov_out)
          for (int j = 0; j < 100; ++j) A.cov_out[pq * 100 + j] = 0.0f;
        map_retired(A, pq);
        continue;
      }
#pragma unroll
      for (int j = 0; j < 10; ++j) Mt[j * kWsSlotsN] = m[j];
      pix = pq;
      sIt[slot] = 0;
      sEps[slot] = A.eps0;
      sFlags[slot] = kFlagFresh;
      return;
    }
  };

  next_pixel();
  sPix[slot] = pix;
  bool any = __any_sync(0xffffffffu, pix >= 0);
  if (!any && lane == 0) fin[b] = 1;
  __syncwarp();
  ws_arrive(bar_empty + 8 * b);
  if (!any) return true;
  uint32_t pf = 0u;
  for (;;) {
    if (!ws_wait(bar_full + 8 * b, pf)) return false;
    pf ^= 1u;
    __syncwarp();
    tc_after();
    __syncwarp();
    // unit-S1 Stokes of every observable (warp-wide loads)
    uint32_t y0[NOBS];
    {
      uint32_t (&ya)[8] = *reinterpret_cast<uint32_t(*)[8]>(y0);
      uint32_t (&yb)[8] = *reinterpret_cast<uint32_t(*)[8]>(y0 + 8);
      uint32_t (&yc)[8] = *reinterpret_cast<uint32_t(*)[8]>(y0 + 16);
      tm_ld8(tc + (uint32_t)(4 * NF * kWsGroup), ya);
      tm_ld8(tc + (uint32_t)(4 * NF * kWsGroup + 8), yb);
      tm_ld8(tc + (uint32_t)(4 * NF * kWsGroup + 16), yc);
      tm_wait24(ya, yb, yc);
    }
    const bool live = pix >= 0;
    const long long px = live ? pix : 0;  // idle lanes read pixel 0's data and drop it
    const float* o = A.obs + px * NOBS;
    const float* wv = weight_row(A, px, NOBS);
    bool accept = false, retire = false, keepA = false;
    int status = VFISV_PIX_MAXITER;
    double c2 = 0.0;
    float c2p = 1.0f, s2p = 0.0f, mus1 = 0.0f, s0 = 0.0f;
    if (live) {
      int it = sIt[slot], fl = sFlags[slot];
      double eps = sEps[slot];
      const double chi2b = sChi[slot];
      // ---- model, residual and chi-square (Eq. 1, FP64) ----
      sincosf(2.0f * Mt[2 * kWsSlotsN] * kDeg, &s2p, &c2p);
      mus1 = A.lk.mu * Mt[8 * kWsSlotsN];
      s0 = Mt[7 * kWsSlotsN];
      float syn[NOBS];
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        const float q0 = __uint_as_float(y0[NF + k]), u0 = __uint_as_float(y0[2 * NF + k]);
        syn[k] = fmaf(s0, tau[k], mus1 * __uint_as_float(y0[k]));
        syn[NF + k] = mus1 * fmaf(c2p, q0, -s2p * u0);
        syn[2 * NF + k] = mus1 * fmaf(s2p, q0, c2p * u0);
        syn[3 * NF + k] = mus1 * __uint_as_float(y0[3 * NF + k]);
      }
      c2 = 0.0;
#pragma unroll
      for (int j = 0; j < NOBS; ++j) {
        const double r = (double)(o[j] - syn[j]);
        c2 = fma((double)wv[j] * r, r, c2);
      }
      c2 /= (double)dof;
      atomicAdd(&cnt[0], 1ull);
      atomicAdd(&cnt[3], (unsigned long long)nrows);
      double rel_acc = INFINITY;
      if (fl & kFlagFresh) {
        accept = isfinite(c2);
        if (!accept) {
          retire = true;
          status = VFISV_PIX_NAN_STATE;
        }
      } else {
        ++it;
        accept = isfinite(c2) && c2 < chi2b;
        const double eps_used = eps;
        eps = eps_update(eps_used, accept);
        bool conv = false, stall = false;
        if (accept) {
          const double rel = (chi2b - c2) / chi2b;
          rel_acc = rel;
          conv = rel < A.conv_rtol && eps_used <= A.conv_eps;
        } else {
          stall = eps >= 1e12;
        }
        if (conv || stall) {
          retire = true;
          status = conv ? VFISV_PIX_CONVERGED : VFISV_PIX_STALLED;
        }
        if (accept) atomicAdd(&cnt[1], 1ull);
      }
      fl &= ~kFlagFresh;
      if (accept) {
        // Hessian reuse (Sec. 4.4): this and the previous accepted step both
        // close to the minimum -> keep J^T W J, rebuild J^T W r only
        const bool nr = rel_acc < A.hess_reuse;
        keepA = nr && (fl & kFlagNear);
        fl = nr ? (fl | kFlagNear) : (fl & ~kFlagNear);
      }
      if (!retire && it >= A.max_iter) retire = true;  // status stays MAXITER
      sIt[slot] = it;
      sEps[slot] = eps;
      sFlags[slot] = fl;
      if (accept) sChi[slot] = c2;
    }
    // ---- J^T W J and J^T W r at an accepted model (compensated FP32); the
    // whole warp takes part in the tensor-memory loads ----
    __syncwarp();
    if (__any_sync(0xffffffffu, accept)) {
      // rows from tensor memory: the next observable's two loads are in
      // flight while the current one is summed
      struct {
        uint32_t tc;
        const float* o;
        const float* wv;
        uint32_t ra[8], rb[8];
        ObsRead<NF> ov;
        __device__ void issue(int k, int s) {
          tm_ld8(tc + (uint32_t)((k * 4 + obs_sa(s)) * kWsGroup), ra);
          tm_ld8(tc + (uint32_t)((k * 4 + obs_sb(s)) * kWsGroup), rb);
          ov.issue(o, wv, k, s);
        }
        __device__ void take(int, int, ObsRows& rw) {
          rw.obs = ov.o;
          rw.w = ov.w;
          tm_wait16(ra, rb);
#pragma unroll
          for (int r = 0; r < kRows; ++r) {
            rw.a[r] = __uint_as_float(ra[r]);
            rw.b[r] = __uint_as_float(rb[r]);
          }
        }
      } fetch{tc, o, wv, {}, {}, {}};
      const RowScale R = row_scale(A.lk, live ? Mt[3 * kWsSlotsN] : 1.0f,
                                   live ? Mt[4 * kWsSlotsN] : 1.0f);
      build_normal_equations<NF, NP, false, true>(
          fetch, tau, scr, ns, mus1, c2p, s2p, s0, 1.0f, A.lk.mu, R, keepA, accept);
    }
    if (live) {
      if (accept) {
#pragma unroll
        for (int j = 0; j < 10; ++j) M[j * kWsSlotsN] = Mt[j * kWsSlotsN];
      }
      if (retire) {
        const bool nan = status == VFISV_PIX_NAN_STATE;
        const float* src = nan ? Mt : M;
        for (int j = 0; j < 10; ++j) A.params_out[pix * 10 + j] = src[j * kWsSlotsN];
        A.chi2_out[pix] = (float)(nan ? c2 : sChi[slot]);
        A.iters_out[pix] = sIt[slot];
        A.status_out[pix] = status;
        if (A.cov_out) {
          // the covariance itself is computed by covariance_kernel for all
          // pixels at once; here the pixel's J^T W J is parked in its row
          float* cv = A.cov_out + pix * 100;
          if (nan) {
            for (int j = 0; j < 100; ++j) cv[j] = 0.0f;
          } else {
            constexpr int NPK4 = (NPK + 3) & ~3;
            float v[NPK4];
#pragma unroll
            for (int j = 0; j < NPK4; ++j) v[j] = (j < NPK) ? scr[(int64_t)j * ns] : 0.0f;
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
        map_retired(A, pix);
        atomicAdd(&cnt[2], 1ull);
        next_pixel();
      } else {
        // ---- next trial model: FP64 damped solve (Eqs. 3-5) ----
        double d[NP];
        damped_step_fp64_body<NP, true>(scr, ns, A.free_mask, sEps[slot], d);
        float m[10];
#pragma unroll
        for (int j = 0; j < NP; ++j) m[j] = (float)((double)M[j * kWsSlotsN] + d[j]);
        m[9] = 1.0f;
        apply_bounds(m);
#pragma unroll
        for (int j = 0; j < 10; ++j) Mt[j * kWsSlotsN] = m[j];
      }
    }
    sPix[slot] = pix;
    any = __any_sync(0xffffffffu, pix >= 0);
    if (!any && lane == 0) fin[b] = 1;
    tc_before();
    __syncwarp();
    ws_arrive(bar_empty + 8 * b);
    if (!any) return true;
  }
}

template <int NF>
__global__ void __launch_bounds__(kWsThreadsN, 1) invert_ws_kernel(InvertArgs A) {
  extern __shared__ __align__(16) float smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int tabf = table_floats(NF, A.nlam);
  const WsSmem L(tabf);
  char* base = reinterpret_cast<char*>(smem);
  float* tab = smem;
  float* sMt = reinterpret_cast<float*>(base + L.mt);
  float* sM = reinterpret_cast<float*>(base + L.m);
  float* sScr = reinterpret_cast<float*>(base + L.scr);
  long long* sPix = reinterpret_cast<long long*>(base + L.pix);
  double* sEps = reinterpret_cast<double*>(base + L.eps);
  double* sChi = reinterpret_cast<double*>(base + L.chi2);
  int* sIt = reinterpret_cast<int*>(base + L.it);
  int* sFlags = reinterpret_cast<int*>(base + L.flags);
  int* fin = reinterpret_cast<int*>(base + L.fin);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(base + L.cnt);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(base + L.tslot);
  const uint32_t bar_full = smem_u32(base + L.bars), bar_empty = bar_full + 8 * kWsBatches;
  if (tid == 0) {
    for (int i = 0; i < 2 * kWsBatches; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_full + 8 * i), "r"(32)
                   : "memory");
  }
  if (tid < kWsBatches) fin[tid] = 0;
  if (tid < 4) cnt[tid] = 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kWsTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the table copy's barrier also publishes the initialisation above
  const bool loaded =
      tma_load_table(tab, A.table, (uint32_t)(tabf * sizeof(float)),
                     reinterpret_cast<uint64_t*>(base + L.tbar), A.err);
  tc_before();
  const bool ok = __syncthreads_and(loaded) != 0;
  tc_after();
  const uint32_t tmem = *tslot;
  const int nrows = table_rows(tab, NF, A.nlam);
  bool good = true;
  if (ok) {
    if (warp < 4) {
      asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kWsProdRegs));
      good = ws_producer<NF>(A, warp, tmem + ((uint32_t)(32 * warp) << 16), tab, nrows, sMt,
                             sPix, fin, bar_full, bar_empty);
    } else {
      asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kWsConsRegs));
      const int b = warp - 4;  // batch: producer b % 4, its batch b / 4
      const uint32_t tc = tmem + ((uint32_t)(32 * (b & 3)) << 16) +
                          ((b >> 2) ? (uint32_t)kWsBatchCols : 0u);
      good = ws_consumer<NF>(A, b, tc, tab, nrows, sMt, sM, sScr, sPix, sEps, sChi, sIt, sFlags,
                             fin, cnt, bar_full, bar_empty);
    }
  }
  if (!good) atomicExch(A.err, kDevErrWsWait);
  tc_before();
  __syncthreads();
  if (warp == 0) {
    tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kWsTmemCols)
                 : "memory");
  }
  if (A.counters && tid < 4) atomicAdd(A.counters + tid, cnt[tid]);
}

}  // namespace

cudaError_t invert_ws_set_constants(const Weideman& W) {
  return cudaMemcpyToSymbol(c_Wws, &W, sizeof(W));
}

size_t invert_ws_smem_bytes(int nlam) { return WsSmem(table_floats(6, nlam)).total; }

cudaError_t invert_ws_slots(int nlam, int64_t npix, int64_t* nslots, int* grid, size_t* smem) {
  const size_t sm = invert_ws_smem_bytes(nlam);
  cudaError_t e = cudaFuncSetAttribute(invert_ws_kernel<6>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  nsm = sm_budget(nsm);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, invert_ws_kernel<6>, kWsThreadsN, sm);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorLaunchOutOfResources;
  // setmaxnreg moves registers within the CTA's launch allocation: the
  // producers' raise waits for registers the consumers' drop frees, so the
  // split must fit the registers the kernel is launched with
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, invert_ws_kernel<6>);
  if (e != cudaSuccess) return e;
  if ((int64_t)fa.numRegs * kWsThreadsN <
      (int64_t)32 * (4 * kWsProdRegs + kWsBatches * kWsConsRegs))
    return cudaErrorInvalidConfiguration;
  int64_t g = nsm;  // one CTA per SM (it holds all of the SM's tensor memory)
  const int64_t need = (npix + kWsSlotsN - 1) / kWsSlotsN;
  if (need < g) g = need;
  if (g < 1) g = 1;
  *grid = (int)g;
  *smem = sm;
  *nslots = g * kWsSlotsN;
  return cudaSuccess;
}

cudaError_t launch_invert_ws(const InvertArgs& a, int grid, size_t smem, cudaStream_t s) {
  invert_ws_kernel<6><<<grid, kWsThreadsN, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace vfisv
