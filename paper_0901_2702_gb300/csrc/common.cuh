// Shared device helpers: the filter/wavelength table staged into shared
// memory by a TMA bulk copy, and kernel launch declarations.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "me_device.cuh"
#include "vfisv.h"

namespace vfisv {

// SMs the persistent launches of the calling handle may use (0: all); set
// per call from the handle (vfisv_set_sm_limit), read by the grid sizing.
extern thread_local int t_sm_limit;
inline int sm_budget(int nsm) { return (t_sm_limit > 0 && t_sm_limit < nsm) ? t_sm_limit : nsm; }

// Device error codes written to the handle's error word.
enum : int {
  kDevErrNone = 0,
  kDevErrTableWait = 1,
  kDevErrNnWait = 2,
  kDevErrPoolWait = 3,
  kDevErrWsWait = 4,  // a hand-off wait of the warp-specialised LM kernel gave up
};

// Filter table layout in global and shared memory: nlam rows of `stride`
// floats {T_0(x_i), ..., T_{nf-1}(x_i), x_i, pad...}, then one row holding
// tau_k = sum_i T_k(x_i).  stride = round_up(nf + 1, 4), so a row is a whole
// number of 16-byte vectors.  Only the first table_rows() rows are used: the
// packing leaves out grid points where every filter weight is negligible
// (synth.cu) and records the count in the last float of the tau row.
__host__ __device__ inline int table_stride(int nf) { return ((nf + 1) + 3) & ~3; }
__host__ __device__ inline int table_floats(int nf, int nlam) {
  return (nlam + 1) * table_stride(nf);
}
__device__ __forceinline__ int table_rows(const float* tab, int nf, int nlam) {
  const int S = table_stride(nf);
  return __float_as_int(tab[(size_t)nlam * S + S - 1]);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Copy `bytes` (multiple of 16, both addresses 16-byte aligned) from global
// to this CTA's shared memory with one TMA bulk copy completing on an
// mbarrier.  Every thread waits, with an iteration bound; returns false and
// flags `err` if the copy did not complete in time.
__device__ inline bool tma_load_table(float* sdst, const float* gsrc, uint32_t bytes,
                                      uint64_t* mbar, int* err) {
  const uint32_t bar = smem_u32(mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(smem_u32(sdst)),
        "l"(gsrc), "r"(bytes), "r"(bar)
        : "memory");
  }
  uint32_t done = 0;
  const long long t0 = clock64();
  for (int it = 0; it < (1 << 22) && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(0)
        : "memory");
    if (!done && clock64() - t0 > (1ll << 31)) break;  // ~1 s at 2 GHz
  }
  if (!done) {
    atomicExch(err, kDevErrTableWait);
    // give the copy in flight a last bounded chance to land before exit
    for (int it = 0; it < (1 << 20) && !done; ++it) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(bar), "r"(0)
          : "memory");
    }
    return false;
  }
  return true;
}

// Read one table row: the NF filter weights and the wavelength offset.
template <int NF>
__device__ __forceinline__ float load_row(const float* row, float (&T)[NF]) {
  constexpr int S = ((NF + 1) + 3) & ~3;
  float v[S];
#pragma unroll
  for (int j = 0; j < S; j += 4) {
    const float4 q = *reinterpret_cast<const float4*>(row + j);
    v[j] = q.x;
    v[j + 1] = q.y;
    v[j + 2] = q.z;
    v[j + 3] = q.w;
  }
#pragma unroll
  for (int k = 0; k < NF; ++k) T[k] = v[k];
  return v[NF];
}

// ---------------------------------------------------------------------------
// Host launchers (one translation unit each).

struct SynthArgs {
  const float* params;
  int64_t npix;
  const float* table;  // packed filter table in global memory
  int nlam;
  float* stokes;
  int* err;
  Weideman W;
  LineK lk;
};

struct InvertArgs {
  const float* obs;
  const float* w;
  int64_t w_stride;  // 4*nf when weights are per pixel, else 0
  const float* init; // may be null: standard guess
  const float* table;
  int nlam;
  int64_t npix;              // pixel count (upper bound when npix_dev is set)
  const int64_t* npix_dev;   // optional device-side count (<= npix)
  float* params_out;
  float* chi2_out;
  int32_t* iters_out;
  int32_t* status_out;
  float* cov_out;    // may be null
  float* scratch;    // [kScratchPerSlot][nslots]
  int64_t nslots;
  unsigned long long* queue;
  int* err;
  Weideman W;
  LineK lk;
  int max_iter;
  uint32_t free_mask;
  int nfree;
  double conv_rtol;
  double conv_eps;
  double eps0;
  double hess_reuse = 0.0;   // Hessian reuse threshold (Sec. 4.4), 0 = off
  int fast_solve = 0;        // 1: double-float solve, compensated FP32 chi2
  // batched maps (the serving mix): map m holds pixels map_off[m] ..
  // map_off[m+1]-1 and its weight row w + m * nobs; each map's completion
  // (global timer, ns) goes to map_t[m] when its last pixel retires
  const int64_t* map_off = nullptr;
  int nmaps = 0;
  unsigned long long* map_done = nullptr;
  unsigned long long* map_t = nullptr;
  int restarts = 0;          // randomised restarts (Sec. 4.2): trigger bit mask, 0 = off
  uint64_t seed = 0;         // key of the restart perturbations
  char* rs_state = nullptr;  // restarts: per-slot state, layout RestartState
  // optional list of the pixels to invert: queue position q inverts pixel
  // pix_list[q] (q < *npix_dev); the others are not touched
  const int64_t* pix_list = nullptr;
  // optional work counters, added to by every CTA when it exits:
  // [0] fused passes (each trial model, plus the starting model),
  // [1] accepted trials (each followed by a J^T W J build), [2] pixels
  // retired, [3] wavelength points evaluated (passes x table rows used)
  unsigned long long* counters = nullptr;
};

constexpr int kScratchPerSlot = 45 + 9;  // packed J^T W J and J^T W r
constexpr int kScratchPerSlotAlpha = 55 + 10;  // the same with the filling factor free

// Map of a pixel in a batch (binary search over the prefix offsets).
__device__ __forceinline__ int map_of(const int64_t* off, int nmaps, int64_t pix) {
  int lo = 0, hi = nmaps;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= pix) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ const float* weight_row(const InvertArgs& A, int64_t pix, int nobs) {
  if (A.map_off) return A.w + (int64_t)map_of(A.map_off, A.nmaps, pix) * nobs;
  return A.w + pix * A.w_stride;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Count a retired pixel of a batch; the map's last one stamps its time.
__device__ __forceinline__ void map_retired(const InvertArgs& A, int64_t pix) {
  if (!A.map_done) return;
  const int m = map_of(A.map_off, A.nmaps, pix);
  const unsigned long long size =
      (unsigned long long)(__ldg(A.map_off + m + 1) - __ldg(A.map_off + m));
  if (atomicAdd(A.map_done + m, 1ull) + 1ull == size) A.map_t[m] = global_ns();
}

// Per-slot state of the randomised restarts, structure of arrays over the
// slots: FP64 [2][ns] (best chi2, initial chi2), FP32 [64][ns] (J^T W J,
// J^T W r and the model at the best chi2), int [3][ns] (failed trials in a
// row, restart count, flags).
constexpr int kRsDoubles = 2, kRsFloats = kScratchPerSlot + 10, kRsInts = 3;
constexpr size_t kRsBytesPerSlot = 8 * kRsDoubles + 4 * kRsFloats + 4 * kRsInts;
struct RestartState {
  double* chi2;  // [2][ns]
  float* f;      // [64][ns]
  int* i;        // [3][ns]
  __host__ __device__ RestartState(char* base, int64_t ns)
      : chi2(reinterpret_cast<double*>(base)),
        f(reinterpret_cast<float*>(base + 8 * kRsDoubles * ns)),
        i(reinterpret_cast<int*>(base + (8 * kRsDoubles + 4 * kRsFloats) * ns)) {}
};
constexpr int kRestartAtConvergence = 1, kRestartA = 2, kRestartB = 4;

cudaError_t launch_pack_table(const float* filters, int nf, const float* wl, int nlam,
                              float* table, cudaStream_t s);
cudaError_t launch_synth(const SynthArgs& a, int nf, cudaStream_t s);
// Persistent LM kernel: launch shape for `npix` pixels with *block threads
// per CTA (64, 128 or 256; anything else selects 128) and *tpp threads per
// pixel (1, 2 or 4; anything else selects 1), both written back as used
// (restarts and a free filling factor take 128 x 1), and the number of
// resident pixel slots (the scratch it needs): grid x block / tpp.
cudaError_t invert_slots(int nf, int nlam, int64_t npix, int restarts, int fast_solve,
                         int alpha_free, int64_t* nslots, int* grid, int* block, int* tpp,
                         size_t* smem);
cudaError_t launch_restart_perturb(const float* in, int64_t n, int64_t pix0, int k,
                                   uint32_t free_mask, uint64_t seed, float* out, cudaStream_t s);
// Upload the Weideman coefficients to the LM kernel's constant bank on the
// current device (once per device).
cudaError_t invert_set_constants(const Weideman& W);
// The warp-specialised LM kernel (invert_ws.cu): CTAs of kInvWsBlock threads
// (one producer warpgroup, two consumer warpgroups), 256 pixel slots each,
// one per SM; the default configuration only (6 filters, FP64 solve, no
// restarts, filling factor held).
constexpr int kInvWsBlock = 384;
cudaError_t invert_ws_set_constants(const Weideman& W);
cudaError_t invert_ws_slots(int nlam, int64_t npix, int64_t* nslots, int* grid, size_t* smem);
cudaError_t launch_invert_ws(const InvertArgs& a, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_covariance(float* cov, const int32_t* status, int64_t npix,
                              const int64_t* npix_dev, uint32_t free_mask, int fast_solve,
                              cudaStream_t s);
cudaError_t launch_invert(const InvertArgs& a, int nf, int grid, int block, int tpp, size_t smem,
                          cudaStream_t s);

// voigt.cu: bulk Voigt/Faraday-Voigt evaluation and the Taylor table.
size_t voigt_table_bytes();
cudaError_t launch_voigt_table(const Weideman& W, void* tab, cudaStream_t s);
cudaError_t launch_voigt(int method, const Weideman& W, const void* tab, const float* a,
                         const float* u, int64_t n, float* H, float* F, cudaStream_t s);

// wide.cu: inputs with many narrow instrument profiles (up to 128 samples
// per Stokes parameter, bands of up to 32 fine points, up to 1024 fine
// points), one pixel per warp.  The compacted table (wide_table_bytes) is
// built by launch_wide_pack, which sets *err to VFISV_E_UNSUPPORTED when a
// band is wider than the kernels take.
bool wide_supported(int nf, int nlam);
size_t wide_table_bytes(int nf, int nlam);
cudaError_t launch_wide_pack(const float* filters, int nf, const float* wl, int nlam,
                             float* table, int* err, cudaStream_t s);
cudaError_t launch_wide_synth(const float* params, int64_t npix, const float* table, int nf,
                              int nlam, float* stokes, int* err, const Weideman& W,
                              const LineK& lk, cudaStream_t s);
cudaError_t launch_wide_invert(const InvertArgs& a, int nf, cudaStream_t s);

// prep.cu: initial models from the filtergrams (Sec. 5); `geom` is device
// scratch of filter_geom_bytes()
size_t filter_geom_bytes();
cudaError_t launch_weak_field(const float* obs, int64_t npix, const int64_t* npix_dev,
                              const float* filters, int nf, const float* wl, int nlam,
                              const LineK& lk, int mode, float pol_thr, void* geom, float* init,
                              float* pol_out, cudaStream_t s);
// prep.cu: batched maps -- a call's start stamp (global timer, ns) and the
// per-map latency in ms from it
cudaError_t launch_stamp(unsigned long long* t, cudaStream_t s);
cudaError_t launch_map_latency(const unsigned long long* t_done, const unsigned long long* t0,
                               int nmaps, float* ms, cudaStream_t s);
// prep.cu: Eq. 14-15 weights
cudaError_t launch_limb_weights(const float* obs, const float* mu, int64_t npix, int nf,
                                float ic0, const float* sigma4, float* w, cudaStream_t s);

}  // namespace vfisv
