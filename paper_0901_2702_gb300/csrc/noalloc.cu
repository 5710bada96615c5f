// vfisv_invert_noalloc: the Levenberg-Marquardt inversion for callers that
// must not allocate device memory.  The kernel's scratch (per-slot normal
// equations, the work-queue counter, the error word and the packed filter
// table) lives in one fixed array compiled into this library instead of a
// handle's workspace.
#include <math.h>

#include <atomic>
#include <mutex>

#include "common.cuh"
#include "vfisv.h"

using namespace vfisv;

namespace {

// Layout of the fixed scratch array (bytes):
//   [0, 256)                 error word (int) and work-queue counter (u64 at 64)
//   [256, 256 + kTableMax)   packed filter/wavelength table, up to 4096 wavelengths
//   [..., + kSlotBytes)      54 floats of J^T W J / J^T W r per pixel slot
constexpr int kMaxNlam = VFISV_NOALLOC_MAX_NLAM;
constexpr int64_t kMaxSlots = VFISV_NOALLOC_MAX_SLOTS;
constexpr size_t kHead = 256;
constexpr size_t kTableMax = ((size_t)(kMaxNlam + 1) * 8 * sizeof(float) + 255) & ~(size_t)255;
constexpr size_t kSlotBytes = (size_t)kScratchPerSlot * kMaxSlots * sizeof(float);
constexpr size_t kScratchBytes = kHead + kTableMax + kSlotBytes;
static_assert(kScratchBytes == VFISV_NOALLOC_SCRATCH_BYTES, "scratch size in vfisv.h");

// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device ordinal, filled on the first call made
// with that device current (the name g_scratch in host code is only a host-side
// stand-in and must never be passed to a kernel).  First calls from several
// host threads are serialised by g_setup; later calls read the published
// address without locking.
constexpr int kMaxDevices = 64;
std::atomic<void*> g_addr[kMaxDevices] = {};
std::mutex g_setup;
Weideman g_W{};
std::once_flag g_W_once;

// Weideman (1994) coefficients as the handle path builds them: trapezoidal
// Fourier coefficients of (L^2 + t^2) exp(-t^2), t = L tan(theta/2), in
// double precision.  Host-only, computed once per process (any thread).
const Weideman& coefficients() {
  std::call_once(g_W_once, [] {
    const int N = kWeidN, M = 64 * N;
    const double L = sqrt(N / sqrt(2.0)), pi = 3.14159265358979323846;
    g_W.L = (float)L;
    g_W.a[0] = 0.0f;
    for (int n = 1; n <= N; ++n) {
      double s = 0.0;
      for (int j = 1; j < M; ++j) {
        const double th = -pi + 2.0 * pi * j / M, t = L * tan(0.5 * th);
        s += (L * L + t * t) * exp(-t * t) * cos(n * th);
      }
      g_W.a[n] = (float)(s / M);
    }
  });
  return g_W;
}

int setup(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return VFISV_E_ARG;
  void* p = g_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    std::lock_guard<std::mutex> lock(g_setup);
    p = g_addr[dev].load(std::memory_order_relaxed);
    if (!p) {
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return VFISV_E_CUDA;
      }
      // error word starts clear; the Weideman coefficients of the LM kernel's
      // constant bank are uploaded for this device
      if (cudaMemset(p, 0, kHead) != cudaSuccess) return VFISV_E_CUDA;
      if (invert_set_constants(coefficients()) != cudaSuccess) return VFISV_E_CUDA;
      g_addr[dev].store(p, std::memory_order_release);
    }
  }
  *out = p;
  return VFISV_OK;
}

// This entry point belongs to no handle: its launches may use every SM,
// whatever SM limit a handle call made earlier on this thread left behind.
struct NoSmLimit {
  int saved = t_sm_limit;
  NoSmLimit() { t_sm_limit = 0; }
  ~NoSmLimit() { t_sm_limit = saved; }
};

}  // namespace

extern "C" int vfisv_invert_noalloc(const float* obs, const float* weights,
                                    int32_t weights_per_pixel, const float* filters,
                                    int32_t nfilt, const float* wl_mA, int32_t nlam,
                                    const vfisv_line* line, const float* init,
                                    const vfisv_config* cfg, int64_t npix, float* params_out,
                                    float* chi2_out, int32_t* iters_out, int32_t* status_out,
                                    float* cov_out, void* stream) {
  if (!obs || !weights || !filters || !wl_mA || !cfg || !params_out || !chi2_out ||
      !iters_out || !status_out || !line || !(line->lambda0_A > 0) || !(line->mu > 0) ||
      !isfinite(line->geff))
    return VFISV_E_ARG;
  if (npix < 0 || nfilt < 1 || nlam < 1) return VFISV_E_SIZE;
  if (nlam > kMaxNlam) return VFISV_E_SIZE;  // the fixed table holds 4096 wavelengths
  if (nfilt != 6) return VFISV_E_UNSUPPORTED;
  if (cfg->restarts != 0) return VFISV_E_UNSUPPORTED;  // restart state is not in the fixed array
  if (cfg->wfa_pol != 0.0) return VFISV_E_UNSUPPORTED;  // the weak-field start needs a buffer
  if (cfg->fast_solve != 0 && cfg->fast_solve != 1) return VFISV_E_ARG;
  if (!(cfg->hess_reuse >= 0) || !isfinite(cfg->hess_reuse)) return VFISV_E_ARG;
  if (cfg->max_iter < 0 || (cfg->free_mask & ~0x1FFu) || !(cfg->conv_rtol >= 0) ||
      !(cfg->conv_eps >= 0) || !(cfg->eps0 > 0) || !isfinite(cfg->eps0) ||
      4 * nfilt - __builtin_popcount(cfg->free_mask) <= 0)
    return VFISV_E_ARG;
  if (npix == 0) return VFISV_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VFISV_E_CUDA;
  void* base = nullptr;
  int rc = setup(dev, &base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  NoSmLimit all_sms;

  int64_t nslots = 0;
  int grid = 0, block = 128, tpp = 1;
  size_t smem = 0;
  if (invert_slots(nfilt, nlam, npix, 0, cfg->fast_solve, 0, &nslots, &grid, &block, &tpp,
                   &smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return VFISV_E_CUDA;
  }
  if (nslots > kMaxSlots) {  // fewer resident slots than the GPU could hold: still correct
    grid = (int)(kMaxSlots / block);
    nslots = (int64_t)grid * block;
  }
  char* b = (char*)base;
  float* table = (float*)(b + kHead);
  // the error word and the work-queue counter start at zero on every call
  // (so vfisv_noalloc_check reports this call's device errors only)
  if (cudaMemsetAsync(b, 0, 64 + sizeof(unsigned long long), s) != cudaSuccess)
    return VFISV_E_CUDA;
  if (launch_pack_table(filters, nfilt, wl_mA, nlam, table, s) != cudaSuccess)
    return VFISV_E_CUDA;
  InvertArgs a;
  a.obs = obs;
  a.w = weights;
  a.w_stride = weights_per_pixel ? 4 * nfilt : 0;
  a.init = init;
  a.table = table;
  a.nlam = nlam;
  a.npix = npix;
  a.npix_dev = nullptr;
  a.params_out = params_out;
  a.chi2_out = chi2_out;
  a.iters_out = iters_out;
  a.status_out = status_out;
  a.cov_out = cov_out;
  a.scratch = (float*)(b + kHead + kTableMax);
  a.nslots = nslots;
  a.queue = (unsigned long long*)(b + 64);
  a.err = (int*)b;
  a.W = coefficients();
  a.lk.cB = (float)(4.66685e-10 * line->geff * line->lambda0_A * line->lambda0_A);
  a.lk.cv = (float)(line->lambda0_A * 1.0e3 / 299792.458);
  a.lk.mu = (float)line->mu;
  a.max_iter = cfg->max_iter;
  a.free_mask = cfg->free_mask;
  a.nfree = __builtin_popcount(cfg->free_mask);
  a.conv_rtol = cfg->conv_rtol;
  a.conv_eps = cfg->conv_eps;
  a.eps0 = cfg->eps0;
  a.hess_reuse = cfg->hess_reuse;
  a.fast_solve = cfg->fast_solve;
  if (launch_invert(a, nfilt, grid, block, tpp, smem, s) != cudaSuccess) return VFISV_E_CUDA;
  if (cov_out &&
      launch_covariance(cov_out, status_out, npix, nullptr, cfg->free_mask, cfg->fast_solve, s) !=
          cudaSuccess)
    return VFISV_E_CUDA;
  return VFISV_OK;
}

extern "C" int vfisv_noalloc_check(void* stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VFISV_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return VFISV_E_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return VFISV_E_CUDA;
  void* p = g_addr[dev].load(std::memory_order_acquire);
  if (!p) return VFISV_OK;  // no call on this device yet
  int err = 0;
  if (cudaMemcpy(&err, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return VFISV_E_CUDA;
  if (err == 0) return VFISV_OK;
  if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return VFISV_E_CUDA;
  return VFISV_E_DEVICE;
}
