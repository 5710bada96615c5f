// C ABI of libvfisv.so: argument checks, host/device pointer staging,
// workspaces, and the Weideman coefficients.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "nn.cuh"
#include "vfisv.h"

using namespace vfisv;

namespace vfisv {
thread_local int t_sm_limit = 0;  // from the calling handle (set_device)
}  // namespace vfisv

struct vfisv_handle {
  int device = 0;
  Weideman W{};
  void* ws = nullptr;      // device workspace: error word, queue, table, scratch
  size_t ws_bytes = 0;
  void* stage = nullptr;   // device staging for host buffers
  size_t stage_bytes = 0;
  void* nnws = nullptr;    // network activations, gradients, optimiser state
  size_t nnws_bytes = 0;
  void* mixws = nullptr;   // mixed inversion: guesses, gathered pixels, 2nd run
  size_t mixws_bytes = 0;
  int lm_block = 128;      // LM threads per CTA (vfisv_autotune)
  int lm_tpp = 1;          // LM threads per pixel (vfisv_autotune)
  void* vtab = nullptr;    // Taylor table of H, F (built on first use)
  void* geom = nullptr;    // filter centres and wing weights of the weak-field init
  size_t geom_bytes = 0;
  void* wfinit = nullptr;  // weak-field initial models of an inversion without init
  size_t wfinit_bytes = 0;
  void* mapws = nullptr;   // batched maps: offsets, counters, stamps (device)
  size_t mapws_bytes = 0;
  int64_t* mapoff_host = nullptr;  // pinned copy of the caller's map offsets
  size_t mapoff_host_bytes = 0;
  bool capturing = false;  // between vfisv_graph_begin and vfisv_graph_end
  // host-buffer pipeline: two device slots, copy-in / copy-out streams and
  // their events (created on first use)
  void* pipe = nullptr;
  size_t pipe_bytes = 0;
  cudaStream_t pipe_in = nullptr, pipe_out = nullptr;
  cudaEvent_t pipe_ev[7] = {};
  int pipe_chunks = 3;     // vfisv_set_pipeline_chunks (0: stage the whole map)
  int sm_limit = 0;        // vfisv_set_sm_limit (0: every SM)
  // work counters of the filter-position LM launches (vfisv_counters):
  // fused passes, accepted trials, pixels retired, wavelength points
  // evaluated (device, u64 each)
  unsigned long long* counters = nullptr;
};

struct vfisv_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

constexpr size_t kAlign = 256;
inline size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Weideman (1994): w(z) = 1/(sqrt(pi)(L - iz)) + 2/(L - iz)^2 sum_{n>=0} a_{n+1} Z^n,
// Z = (L + iz)/(L - iz).  The a_n are the Fourier coefficients of
// f(theta) = (L^2 + t^2) exp(-t^2), t = L tan(theta/2), obtained here by the
// trapezoidal rule on a uniform theta grid (spectrally accurate for this
// smooth periodic f), in double precision.
Weideman weideman_coefficients() {
  Weideman W{};
  const int N = kWeidN;
  const double L = sqrt(N / sqrt(2.0));
  const int M = 64 * N;
  const double pi = 3.14159265358979323846;
  std::vector<double> th(M), f(M);
  for (int j = 0; j < M; ++j) {
    th[j] = -pi + 2.0 * pi * j / M;
    if (j == 0) {
      f[j] = 0.0;  // t = -infinity
    } else {
      const double t = L * tan(0.5 * th[j]);
      f[j] = (L * L + t * t) * exp(-t * t);
    }
  }
  W.L = (float)L;
  W.a[0] = 0.0f;
  for (int n = 1; n <= N; ++n) {
    double s = 0.0;
    for (int j = 0; j < M; ++j) s += f[j] * cos(n * th[j]);
    W.a[n] = (float)(s / M);
  }
  return W;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Set while a handle is capturing a graph: workspaces must not grow then
// (a cudaMalloc / cudaFree would not be recorded and would synchronise).
thread_local bool t_capturing = false;

int grow(void** buf, size_t* have, size_t need) {
  if (*have >= need) return VFISV_OK;
  if (t_capturing) return VFISV_E_CAPTURE;
  if (*buf) {
    cudaDeviceSynchronize();
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
  }
  if (cudaMalloc(buf, need) != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return VFISV_E_NOMEM;
  }
  // a workspace starts with the device error word: clear it
  if (cudaMemset(*buf, 0, need < 256 ? need : 256) != cudaSuccess) return VFISV_E_CUDA;
  *have = need;
  return VFISV_OK;
}

LineK line_constants(const vfisv_line* l) {
  LineK k;
  // Eq. 7: dlambda_B [mA] = 4.66685e-10 g_eff lambda0[A]^2 B[G]
  k.cB = (float)(4.66685e-10 * l->geff * l->lambda0_A * l->lambda0_A);
  // Doppler: lambda0 v / c with lambda0 in mA and c in km/s
  k.cv = (float)(l->lambda0_A * 1.0e3 / 299792.458);
  k.mu = (float)l->mu;
  return k;
}

bool line_ok(const vfisv_line* l) {
  return l && isfinite(l->lambda0_A) && l->lambda0_A > 0 && isfinite(l->geff) &&
         isfinite(l->mu) && l->mu > 0;
}

// A set of caller buffers, each either device memory (used in place) or
// host memory (staged through the handle's staging area).
struct Buf {
  const void* user;
  size_t bytes;
  bool out;
  bool host;
  void* dev;
};

struct Staging {
  std::vector<Buf> bufs;
  void add(const void* p, size_t bytes, bool out) {
    bufs.push_back(Buf{p, bytes, out, p && !is_device_ptr(p), nullptr});
  }
  int prepare(vfisv_handle* h, cudaStream_t s) {
    size_t need = 0;
    for (auto& b : bufs)
      if (b.host && b.bytes) need += up(b.bytes);
    int rc = grow(&h->stage, &h->stage_bytes, need > 0 ? need : 0);
    if (rc) return rc;
    size_t off = 0;
    for (auto& b : bufs) {
      if (!b.user) continue;
      if (!b.host) {
        b.dev = const_cast<void*>(b.user);
        continue;
      }
      b.dev = (char*)h->stage + off;
      off += up(b.bytes);
      if (!b.out && b.bytes &&
          cudaMemcpyAsync(b.dev, b.user, b.bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return VFISV_E_CUDA;
    }
    return VFISV_OK;
  }
  bool any_host() const {
    for (auto& b : bufs)
      if (b.host) return true;
    return false;
  }
  int finish(cudaStream_t s) {
    bool sync = false;
    for (auto& b : bufs)
      if (b.host && b.out && b.bytes) {
        if (cudaMemcpyAsync(const_cast<void*>(b.user), b.dev, b.bytes, cudaMemcpyDeviceToHost,
                            s) != cudaSuccess)
          return VFISV_E_CUDA;
        sync = true;
      }
    if (sync || any_host())
      if (cudaStreamSynchronize(s) != cudaSuccess) return VFISV_E_CUDA;
    return VFISV_OK;
  }
};

// Host-buffer pipeline for per-pixel calls on large maps.  Rows [0, npix)
// run in h->pipe_chunks chunks; each chunk's host inputs are copied in on one
// stream and its host outputs copied back on another, through two device
// slots, while the caller's stream computes the previous chunk -- so the
// host<->device traffic hides behind the inversion.  Only the first chunk's
// copy-in and the last chunk's copy-out stay exposed, so with three or more
// chunks those two are an eighth of the size of the others.  Every per-pixel
// result depends on that pixel alone, so the outputs equal those of one call
// over the whole map.  Device pointers among the rows are used in place.
constexpr int64_t kPipeMinRows = 1 << 20;

struct RowArg {
  const void* user;  // caller pointer (host or device) or null
  size_t row_bytes;  // bytes per pixel
  bool out;
};

template <class Run>
int pipeline_rows_impl(vfisv_handle* h, cudaStream_t s, int64_t npix, RowArg* args, int nargs,
                       Run run);

// On an error the copies already queued still read and write the caller's
// host buffers: let them finish before returning, so the caller may free them.
template <class Run>
int pipeline_rows(vfisv_handle* h, cudaStream_t s, int64_t npix, RowArg* args, int nargs,
                  Run run) {
  const int rc = pipeline_rows_impl(h, s, npix, args, nargs, run);
  if (rc != VFISV_OK) {
    if (h->pipe_in) cudaStreamSynchronize(h->pipe_in);
    if (h->pipe_out) cudaStreamSynchronize(h->pipe_out);
    cudaStreamSynchronize(s);
  }
  return rc;
}

template <class Run>
int pipeline_rows_impl(vfisv_handle* h, cudaStream_t s, int64_t npix, RowArg* args, int nargs,
                       Run run) {
  // chunk boundaries: weights 1/8, 1, ..., 1, 1/8 (uniform below 3 chunks)
  const int nc = h->pipe_chunks;
  std::vector<int64_t> bound(nc + 1);
  const double edge = nc >= 3 ? 0.125 : 1.0, total_w = 2 * edge + (nc - 2);
  double acc = 0.0;
  for (int k = 0; k <= nc; ++k) {
    bound[k] = k == nc ? npix : (int64_t)((double)npix * acc / (nc == 1 ? 1.0 : total_w));
    if (k < nc) acc += (k == 0 || k == nc - 1) ? (nc == 1 ? 1.0 : edge) : 1.0;
  }
  int64_t chunk = 0;
  for (int k = 0; k < nc; ++k) chunk = bound[k + 1] - bound[k] > chunk ? bound[k + 1] - bound[k] : chunk;
  std::vector<bool> host(nargs);
  size_t slot = 0;
  for (int i = 0; i < nargs; ++i) {
    host[i] = args[i].user && !is_device_ptr(args[i].user);
    if (host[i]) slot += up((size_t)chunk * args[i].row_bytes);
  }
  int rc = grow(&h->pipe, &h->pipe_bytes, 2 * slot);
  if (rc) return rc;
  if (!h->pipe_in) {
    if (cudaStreamCreateWithFlags(&h->pipe_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->pipe_out, cudaStreamNonBlocking) != cudaSuccess)
      return VFISV_E_CUDA;
    for (cudaEvent_t& e : h->pipe_ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return VFISV_E_CUDA;
  }
  cudaEvent_t* ev_in = h->pipe_ev + 1;    // chunk's inputs in slot j
  cudaEvent_t* ev_done = h->pipe_ev + 3;  // chunk computed
  cudaEvent_t* ev_free = h->pipe_ev + 5;  // slot j copied out
  // the copies start after the work already queued on the caller's stream
  if (cudaEventRecord(h->pipe_ev[0], s) != cudaSuccess ||
      cudaStreamWaitEvent(h->pipe_in, h->pipe_ev[0], 0) != cudaSuccess ||
      cudaStreamWaitEvent(h->pipe_out, h->pipe_ev[0], 0) != cudaSuccess)
    return VFISV_E_CUDA;
  std::vector<void*> dev(nargs);
  for (int k = 0; k < nc; ++k) {
    const int j = k & 1;
    const int64_t off = bound[k], n = bound[k + 1] - bound[k];
    if (n == 0) continue;
    char* base = (char*)h->pipe + (size_t)j * slot;
    for (int i = 0; i < nargs; ++i) {
      if (!args[i].user) {
        dev[i] = nullptr;
      } else if (!host[i]) {
        dev[i] = (char*)args[i].user + (size_t)off * args[i].row_bytes;
      } else {
        dev[i] = base;
        base += up((size_t)chunk * args[i].row_bytes);
      }
    }
    if (k >= 2 && cudaStreamWaitEvent(h->pipe_in, ev_free[j], 0) != cudaSuccess)
      return VFISV_E_CUDA;
    for (int i = 0; i < nargs; ++i)
      if (host[i] && !args[i].out &&
          cudaMemcpyAsync(dev[i], (const char*)args[i].user + (size_t)off * args[i].row_bytes,
                          (size_t)n * args[i].row_bytes, cudaMemcpyHostToDevice,
                          h->pipe_in) != cudaSuccess)
        return VFISV_E_CUDA;
    if (cudaEventRecord(ev_in[j], h->pipe_in) != cudaSuccess ||
        cudaStreamWaitEvent(s, ev_in[j], 0) != cudaSuccess)
      return VFISV_E_CUDA;
    if ((rc = run(n, dev.data())) != VFISV_OK) return rc;
    if (cudaEventRecord(ev_done[j], s) != cudaSuccess ||
        cudaStreamWaitEvent(h->pipe_out, ev_done[j], 0) != cudaSuccess)
      return VFISV_E_CUDA;
    for (int i = 0; i < nargs; ++i)
      if (host[i] && args[i].out &&
          cudaMemcpyAsync((char*)args[i].user + (size_t)off * args[i].row_bytes, dev[i],
                          (size_t)n * args[i].row_bytes, cudaMemcpyDeviceToHost,
                          h->pipe_out) != cudaSuccess)
        return VFISV_E_CUDA;
    if (cudaEventRecord(ev_free[j], h->pipe_out) != cudaSuccess) return VFISV_E_CUDA;
  }
  if (cudaStreamSynchronize(h->pipe_out) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return VFISV_E_CUDA;
  return VFISV_OK;
}

// Large maps in host memory take the pipeline (not while capturing a graph,
// and not with restarts, whose random draws are keyed by the pixel's index
// within the call).
bool pipeline_host(const vfisv_handle* h, const void* obs, int64_t npix, bool no_restarts) {
  return !h->capturing && no_restarts && h->pipe_chunks > 0 && npix >= kPipeMinRows &&
         !is_device_ptr(obs);
}

// Workspace layout: [err int | queue u64 | pad] [table] [scratch] [restart state]
struct WsLayout {
  size_t err = 0, queue = 64, table = 256, scratch = 0, rs = 0, total = 0;
};

WsLayout layout(int nf, int nlam, int64_t nslots, bool restarts, bool alpha_free = false) {
  WsLayout L;
  size_t tb = (size_t)table_floats(nf, nlam) * sizeof(float);
  if (nf > 8 && wide_table_bytes(nf, nlam) > tb) tb = wide_table_bytes(nf, nlam);
  L.scratch = L.table + up(tb);
  const size_t per = alpha_free ? kScratchPerSlotAlpha : kScratchPerSlot;
  L.rs = L.scratch + up(per * (size_t)nslots * sizeof(float));
  L.total = L.rs + (restarts ? up(kRsBytesPerSlot * (size_t)nslots) : 0);
  return L;
}

int set_device(vfisv_handle* h) {
  t_capturing = h->capturing;
  t_sm_limit = h->sm_limit;
  return cudaSetDevice(h->device) == cudaSuccess ? VFISV_OK : VFISV_E_CUDA;
}


int check_config(const vfisv_config* cfg, int nfilt) {
  if (!cfg) return VFISV_E_ARG;
  if (cfg->max_iter < 0 || (cfg->free_mask & ~0x3FFu) || !(cfg->conv_rtol >= 0) ||
      !(cfg->conv_eps >= 0) || !(cfg->eps0 > 0) || !isfinite(cfg->eps0))
    return VFISV_E_ARG;
  // the filling factor free (bit 9): the FP64 solve without restarts
  if ((cfg->free_mask >> 9) & 1u && (cfg->restarts || cfg->fast_solve)) return VFISV_E_UNSUPPORTED;
  // restart counters are 20 bits wide (each restart costs an iteration)
  if ((cfg->restarts & ~7) || (cfg->restarts && cfg->max_iter >= (1 << 20))) return VFISV_E_ARG;
  if (!(cfg->hess_reuse >= 0) || !isfinite(cfg->hess_reuse)) return VFISV_E_ARG;
  if (!(cfg->wfa_pol >= 0) || !isfinite(cfg->wfa_pol)) return VFISV_E_ARG;
  if (cfg->fast_solve != 0 && cfg->fast_solve != 1) return VFISV_E_ARG;
  if (4 * nfilt - __builtin_popcount(cfg->free_mask) <= 0) return VFISV_E_ARG;
  return VFISV_OK;
}

int check_invert_args(vfisv_handle* h, const float* obs, const float* weights,
                      const float* filters, int32_t nfilt, const float* wl_mA, int32_t nlam,
                      const vfisv_line* line, const vfisv_config* cfg, int64_t npix,
                      const float* params_out, const float* chi2_out, const int32_t* iters_out,
                      const int32_t* status_out) {
  if (!h || !obs || !weights || !filters || !wl_mA || !cfg || !params_out || !chi2_out ||
      !iters_out || !status_out || !line_ok(line))
    return VFISV_E_ARG;
  if (npix < 0 || nfilt < 1 || nlam < 1 || nlam > 4096) return VFISV_E_SIZE;
  if (nfilt != 6 && !(nfilt > 8 && wide_supported(nfilt, nlam))) return VFISV_E_UNSUPPORTED;
  if (nfilt > 8 && cfg &&
      (cfg->restarts || cfg->hess_reuse != 0.0 || cfg->fast_solve ||
       ((cfg->free_mask >> 9) & 1u)))
    return VFISV_E_UNSUPPORTED;  // options of the filter-position kernel only
  return check_config(cfg, nfilt);
}

// Device buffers of one inversion.
struct DevInvert {
  const float *obs = nullptr, *w = nullptr, *filters = nullptr, *wl = nullptr, *init = nullptr;
  int64_t w_stride = 0;
  float *params = nullptr, *chi2 = nullptr, *cov = nullptr;
  int32_t *iters = nullptr, *status = nullptr;
  // batched maps (vfisv_invert_batch)
  const int64_t* map_off = nullptr;
  int nmaps = 0;
  unsigned long long *map_done = nullptr, *map_t = nullptr;
  // invert only the listed pixels (*npix_dev of them) of a map of npix
  const int64_t* pix_list = nullptr;
  // leave each pixel's J^T W J parked in its covariance row (the caller runs
  // the covariance kernel once over the final rows)
  bool park_cov = false;
};

// Pack the filter table, zero the work queue, run the persistent LM kernel
// and the batched covariance, all on stream s.
// Many narrow instrument profiles (spectrograph-shaped inputs): the
// warp-per-pixel kernel, then the batched covariance.
int invert_device_wide(vfisv_handle* h, const DevInvert& d, int nfilt, int nlam,
                       const vfisv_line* line, const vfisv_config* cfg, int64_t npix,
                       const int64_t* npix_dev, cudaStream_t s) {
  WsLayout L = layout(nfilt, nlam, 0, false);
  if (h->ws_bytes < L.total) {
    int rc = grow(&h->ws, &h->ws_bytes, L.total);
    if (rc) return rc;
    if (cudaMemsetAsync(h->ws, 0, 64, s) != cudaSuccess) return VFISV_E_CUDA;
  }
  char* ws = (char*)h->ws;
  float* table = (float*)(ws + L.table);
  int* err = (int*)(ws + L.err);
  const float* init = d.init;
  if (!init && cfg->wfa_pol > 0.0) {
    // start from the weak-field models of the observations (Sec. 5)
    int rc = grow(&h->geom, &h->geom_bytes, filter_geom_bytes());
    if (!rc) rc = grow(&h->wfinit, &h->wfinit_bytes, (size_t)npix * 10 * sizeof(float));
    if (rc) return rc;
    if (launch_weak_field(d.obs, npix, npix_dev, d.filters, nfilt, d.wl, nlam,
                          line_constants(line), 0, 0.0f, h->geom, (float*)h->wfinit, nullptr,
                          s) != cudaSuccess)
      return VFISV_E_CUDA;
    init = (const float*)h->wfinit;
  }
  if (launch_wide_pack(d.filters, nfilt, d.wl, nlam, table, err, s) != cudaSuccess)
    return VFISV_E_CUDA;
  if (cudaMemsetAsync(ws + L.queue, 0, sizeof(unsigned long long), s) != cudaSuccess)
    return VFISV_E_CUDA;
  InvertArgs a;
  a.obs = d.obs;
  a.w = d.w;
  a.w_stride = d.w_stride;
  a.init = init;
  a.table = table;
  a.nlam = nlam;
  a.npix = npix;
  a.npix_dev = npix_dev;
  a.params_out = d.params;
  a.chi2_out = d.chi2;
  a.iters_out = d.iters;
  a.status_out = d.status;
  a.cov_out = d.cov;
  a.scratch = nullptr;
  a.nslots = 0;
  a.queue = (unsigned long long*)(ws + L.queue);
  a.err = err;
  a.W = h->W;
  a.lk = line_constants(line);
  a.max_iter = cfg->max_iter;
  a.free_mask = cfg->free_mask;
  a.nfree = __builtin_popcount(cfg->free_mask);
  a.conv_rtol = cfg->conv_rtol;
  a.conv_eps = cfg->conv_eps;
  a.eps0 = cfg->eps0;
  a.map_off = d.map_off;
  a.nmaps = d.nmaps;
  a.map_done = d.map_done;
  a.map_t = d.map_t;
  if (launch_wide_invert(a, nfilt, s) != cudaSuccess) return VFISV_E_CUDA;
  // the kernel parks each pixel's J^T W J in its covariance row
  if (d.cov && !d.park_cov &&
      launch_covariance(d.cov, d.status, npix, npix_dev, cfg->free_mask, 0, s) !=
                   cudaSuccess)
    return VFISV_E_CUDA;
  return VFISV_OK;
}

int invert_device(vfisv_handle* h, const DevInvert& d, int nfilt, int nlam,
                  const vfisv_line* line, const vfisv_config* cfg, int64_t npix,
                  const int64_t* npix_dev, cudaStream_t s) {
  if (nfilt > 8) return invert_device_wide(h, d, nfilt, nlam, line, cfg, npix, npix_dev, s);
  int64_t nslots = 0;
  int grid = 0, block = h->lm_block, tpp = h->lm_tpp;
  size_t smem = 0;
  const bool alpha_free = (cfg->free_mask >> 9) & 1u;
  if (invert_slots(nfilt, nlam, npix, cfg->restarts, cfg->fast_solve, alpha_free, &nslots, &grid,
                   &block, &tpp, &smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return VFISV_E_CUDA;
  }
  WsLayout L = layout(nfilt, nlam, nslots, cfg->restarts != 0, alpha_free);
  if (h->ws_bytes < L.total) {
    int rc = grow(&h->ws, &h->ws_bytes, L.total);
    if (rc) return rc;
    if (cudaMemsetAsync(h->ws, 0, 64, s) != cudaSuccess) return VFISV_E_CUDA;
  }
  char* ws = (char*)h->ws;
  float* table = (float*)(ws + L.table);
  const float* init = d.init;
  if (!init && cfg->wfa_pol > 0.0) {
    // start from the weak-field models of the filtergrams (Sec. 5)
    int rc = grow(&h->geom, &h->geom_bytes, filter_geom_bytes());
    if (!rc) rc = grow(&h->wfinit, &h->wfinit_bytes, (size_t)npix * 10 * sizeof(float));
    if (rc) return rc;
    if (launch_weak_field(d.obs, npix, npix_dev, d.filters, nfilt, d.wl, nlam,
                          line_constants(line), 0, 0.0f, h->geom, (float*)h->wfinit, nullptr,
                          s) != cudaSuccess)
      return VFISV_E_CUDA;
    init = (const float*)h->wfinit;
  }
  if (launch_pack_table(d.filters, nfilt, d.wl, nlam, table, s) != cudaSuccess)
    return VFISV_E_CUDA;
  if (cudaMemsetAsync(ws + L.queue, 0, sizeof(unsigned long long), s) != cudaSuccess)
    return VFISV_E_CUDA;
  InvertArgs a;
  a.obs = d.obs;
  a.w = d.w;
  a.w_stride = d.w_stride;
  a.init = init;
  a.table = table;
  a.nlam = nlam;
  a.npix = npix;
  a.npix_dev = npix_dev;
  a.params_out = d.params;
  a.chi2_out = d.chi2;
  a.iters_out = d.iters;
  a.status_out = d.status;
  a.cov_out = d.cov;
  a.scratch = (float*)(ws + L.scratch);
  a.nslots = nslots;
  a.queue = (unsigned long long*)(ws + L.queue);
  a.err = (int*)(ws + L.err);
  a.W = h->W;
  a.lk = line_constants(line);
  a.max_iter = cfg->max_iter;
  a.free_mask = cfg->free_mask;
  a.nfree = __builtin_popcount(cfg->free_mask);
  a.conv_rtol = cfg->conv_rtol;
  a.conv_eps = cfg->conv_eps;
  a.eps0 = cfg->eps0;
  a.map_off = d.map_off;
  a.nmaps = d.nmaps;
  a.map_done = d.map_done;
  a.map_t = d.map_t;
  a.restarts = cfg->restarts;
  a.seed = cfg->seed;
  a.hess_reuse = cfg->hess_reuse;
  a.fast_solve = cfg->fast_solve;
  a.rs_state = cfg->restarts ? ws + L.rs : nullptr;
  a.pix_list = d.pix_list;
  a.counters = h->counters;
  if (launch_invert(a, nfilt, grid, block, tpp, smem, s) != cudaSuccess) return VFISV_E_CUDA;
  // with a pixel list the listed pixels lie anywhere in [0, npix): the
  // covariance kernel sweeps the whole map (it skips rows by status)
  if (d.cov && !d.park_cov &&
      launch_covariance(d.cov, d.status, npix, d.pix_list ? nullptr : npix_dev, cfg->free_mask,
                        cfg->fast_solve, s) !=
                   cudaSuccess)
    return VFISV_E_CUDA;
  return VFISV_OK;
}

}  // namespace

extern "C" {

const char* vfisv_strerror(int code) {
  switch (code) {
    case VFISV_OK: return "ok";
    case VFISV_E_ARG: return "invalid argument";
    case VFISV_E_SIZE: return "size out of the supported range";
    case VFISV_E_UNSUPPORTED: return "number of filters not compiled into this kernel";
    case VFISV_E_CUDA: return "CUDA runtime error";
    case VFISV_E_DEVICE: return "a kernel reported an internal error";
    case VFISV_E_NOMEM: return "device workspace allocation failed";
    case VFISV_E_CAPTURE:
      return "a workspace would have to grow during graph capture: make one uncaptured call "
             "with the same sizes first";
    default: return "unknown error";
  }
}

void vfisv_config_default(vfisv_config* c) {
  if (!c) return;
  c->max_iter = 50;
  c->free_mask = 0x1FFu;
  c->conv_rtol = 1e-4;
  c->conv_eps = 1.0;
  c->eps0 = 1.0;
  c->restarts = 0;
  c->seed = 0;
  c->hess_reuse = 0.0;
  c->wfa_pol = 0.0;
  c->fast_solve = 0;
}

int vfisv_create(vfisv_handle** out, int device) {
  if (!out) return VFISV_E_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return VFISV_E_CUDA;
  }
  if (device < 0 || device >= n) return VFISV_E_ARG;
  vfisv_handle* h = new vfisv_handle();
  h->device = device;
  h->W = weideman_coefficients();
  if (set_device(h) != VFISV_OK || invert_set_constants(h->W) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return VFISV_E_CUDA;
  }
  if (cudaMalloc(&h->counters, 4 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(h->counters, 0, 4 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    if (h->counters) cudaFree(h->counters);
    delete h;
    return VFISV_E_NOMEM;
  }
  *out = h;
  return VFISV_OK;
}

int vfisv_counters(vfisv_handle* h, void* stream, uint64_t* out, int32_t reset) {
  if (!h || !out) return VFISV_E_ARG;
  if (set_device(h)) return VFISV_E_CUDA;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return VFISV_E_CUDA;
  unsigned long long c[4] = {0, 0, 0, 0};
  if (cudaMemcpy(c, h->counters, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
    return VFISV_E_CUDA;
  for (int i = 0; i < 4; ++i) out[i] = (uint64_t)c[i];
  if (reset && cudaMemset(h->counters, 0, sizeof(c)) != cudaSuccess) return VFISV_E_CUDA;
  return VFISV_OK;
}

void vfisv_destroy(vfisv_handle* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  if (h->ws) cudaFree(h->ws);
  if (h->counters) cudaFree(h->counters);
  if (h->stage) cudaFree(h->stage);
  if (h->nnws) cudaFree(h->nnws);
  if (h->mixws) cudaFree(h->mixws);
  if (h->vtab) cudaFree(h->vtab);
  if (h->geom) cudaFree(h->geom);
  if (h->wfinit) cudaFree(h->wfinit);
  if (h->mapws) cudaFree(h->mapws);
  if (h->mapoff_host) cudaFreeHost(h->mapoff_host);
  if (h->pipe) cudaFree(h->pipe);
  if (h->pipe_in) cudaStreamDestroy(h->pipe_in);
  if (h->pipe_out) cudaStreamDestroy(h->pipe_out);
  for (cudaEvent_t e : h->pipe_ev)
    if (e) cudaEventDestroy(e);
  delete h;
}

int vfisv_graph_begin(vfisv_handle* h, void* stream) {
  if (!h || !stream || h->capturing) return VFISV_E_ARG;
  if (set_device(h)) return VFISV_E_CUDA;
  if (cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return VFISV_E_CUDA;
  }
  h->capturing = true;
  t_capturing = true;
  return VFISV_OK;
}

int vfisv_graph_end(vfisv_handle* h, void* stream, vfisv_graph** out) {
  if (!h || !stream || !out || !h->capturing) return VFISV_E_ARG;
  *out = nullptr;
  h->capturing = false;
  t_capturing = false;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture((cudaStream_t)stream, &g) != cudaSuccess || !g) {
    cudaGetLastError();
    return VFISV_E_CUDA;
  }
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return VFISV_E_CUDA;
  }
  vfisv_graph* r = new vfisv_graph();
  r->graph = g;
  r->exec = ex;
  *out = r;
  return VFISV_OK;
}

int vfisv_graph_launch(vfisv_graph* g, void* stream) {
  if (!g || !g->exec) return VFISV_E_ARG;
  return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? VFISV_OK : VFISV_E_CUDA;
}

static int count_kernels(cudaGraph_t g, int64_t* count) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return VFISV_E_CUDA;
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return VFISV_E_CUDA;
  for (cudaGraphNode_t node : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(node, &t) != cudaSuccess) return VFISV_E_CUDA;
    if (t == cudaGraphNodeTypeKernel) {
      ++*count;
    } else if (t == cudaGraphNodeTypeGraph) {
      cudaGraph_t child;
      if (cudaGraphChildGraphNodeGetGraph(node, &child) != cudaSuccess) return VFISV_E_CUDA;
      const int rc = count_kernels(child, count);
      if (rc) return rc;
    }
  }
  return VFISV_OK;
}

int vfisv_graph_kernels(const vfisv_graph* g, int64_t* count) {
  if (!g || !g->graph || !count) return VFISV_E_ARG;
  *count = 0;
  return count_kernels(g->graph, count);
}

void vfisv_graph_destroy(vfisv_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

int vfisv_set_sm_limit(vfisv_handle* h, int32_t nsm) {
  if (!h || nsm < 0) return VFISV_E_ARG;
  h->sm_limit = nsm;
  return VFISV_OK;
}

int vfisv_set_pipeline_chunks(vfisv_handle* h, int32_t chunks) {
  if (!h || chunks < 0 || chunks > 64) return VFISV_E_ARG;
  h->pipe_chunks = chunks;
  return VFISV_OK;
}

int vfisv_autotune(vfisv_handle* h, const float* obs, const float* weights,
                   int32_t weights_per_pixel, const float* filters, int32_t nfilt,
                   const float* wl_mA, int32_t nlam, const vfisv_line* line,
                   const vfisv_config* cfg, int64_t npix, int32_t* best_block, int32_t* best_tpp,
                   float* ms_out, void* stream) {
  if (!h || !best_block || h->capturing) return VFISV_E_ARG;
  if (npix < 1) return VFISV_E_SIZE;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // outputs of the trial runs live in the mixed-inversion workspace
  size_t off = 0;
  auto place = [&](size_t bytes) {
    const size_t at = off;
    off += up(bytes);
    return at;
  };
  const size_t o_p = place((size_t)npix * 40), o_c = place((size_t)npix * 4),
               o_i = place((size_t)npix * 4), o_s = place((size_t)npix * 4);
  int rc = grow(&h->mixws, &h->mixws_bytes, off);
  if (rc) return rc;
  char* mw = (char*)h->mixws;
  // threads per CTA x threads per pixel, threads-per-pixel-major, then the
  // warp-specialised kernel (kInvWsBlock threads, one pixel per consumer
  // thread)
  const int cand_b[3] = {64, 128, 256}, cand_t[3] = {1, 2, 4};
  auto shape = [&](int c, int* b, int* t) {
    *b = (c < 9) ? cand_b[c % 3] : kInvWsBlock;
    *t = (c < 9) ? cand_t[c / 3] : 1;
  };
  float best = 0.0f;
  int best_b = 128, best_t = 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int c = 0; c < 10; ++c) {
    shape(c, &h->lm_block, &h->lm_tpp);
    float ms = 0.0f;
    for (int rep = 0; rep < 2; ++rep) {  // the first run warms up
      cudaEventRecord(e0, s);
      rc = vfisv_invert(h, obs, weights, weights_per_pixel, filters, nfilt, wl_mA, nlam, line,
                        nullptr, cfg, npix, (float*)(mw + o_p), (float*)(mw + o_c),
                        (int32_t*)(mw + o_i), (int32_t*)(mw + o_s), nullptr, stream);
      cudaEventRecord(e1, s);
      if (rc) break;
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    if (rc) break;
    if (ms_out) ms_out[c] = ms;
    if (c == 0 || ms < best) {
      best = ms;
      shape(c, &best_b, &best_t);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->lm_block = best_b;
  h->lm_tpp = best_t;
  *best_block = best_b;
  if (best_tpp) *best_tpp = best_t;
  return rc;
}

int vfisv_set_launch_shape(vfisv_handle* h, int32_t block, int32_t tpp) {
  const bool plain = (block == 64 || block == 128 || block == 256) && (tpp == 1 || tpp == 2 || tpp == 4);
  if (!h || !(plain || (block == kInvWsBlock && tpp == 1))) return VFISV_E_ARG;
  h->lm_block = block;
  h->lm_tpp = tpp;
  return VFISV_OK;
}

int vfisv_voigt(vfisv_handle* h, const float* a, const float* u, int64_t n, int32_t method,
                float* H, float* F, void* stream) {
  if (!h || !a || !u || !H || !F || method < 0 || method > 2) return VFISV_E_ARG;
  if (n < 0) return VFISV_E_SIZE;
  if (n == 0) return VFISV_OK;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  if (method > 0 && !h->vtab) {
    size_t have = 0;
    int rc = grow(&h->vtab, &have, voigt_table_bytes());
    if (rc) return rc;
    if (launch_voigt_table(h->W, h->vtab, s) != cudaSuccess) return VFISV_E_CUDA;
  }
  Staging st;
  st.add(a, (size_t)n * sizeof(float), false);
  st.add(u, (size_t)n * sizeof(float), false);
  st.add(H, (size_t)n * sizeof(float), true);
  st.add(F, (size_t)n * sizeof(float), true);
  int rc = st.prepare(h, s);
  if (rc) return rc;
  if (launch_voigt(method, h->W, h->vtab, (const float*)st.bufs[0].dev,
                   (const float*)st.bufs[1].dev, n, (float*)st.bufs[2].dev,
                   (float*)st.bufs[3].dev, s) != cudaSuccess)
    return VFISV_E_CUDA;
  return st.finish(s);
}

int vfisv_init_models(vfisv_handle* h, const float* obs, int64_t npix, const float* filters,
                      int32_t nfilt, const float* wl_mA, int32_t nlam, const vfisv_line* line,
                      float* init_out, float* pol_out, void* stream) {
  if (!h || !obs || !filters || !wl_mA || !init_out || !line_ok(line)) return VFISV_E_ARG;
  if (npix < 0 || nlam < 1 || nlam > 4096) return VFISV_E_SIZE;
  if (nfilt < 3 || nfilt > 128) return VFISV_E_UNSUPPORTED;
  if (npix == 0) return VFISV_OK;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = grow(&h->geom, &h->geom_bytes, filter_geom_bytes());
  if (rc) return rc;
  Staging st;
  st.add(obs, (size_t)npix * 4 * nfilt * sizeof(float), false);
  st.add(filters, (size_t)nfilt * nlam * sizeof(float), false);
  st.add(wl_mA, (size_t)nlam * sizeof(float), false);
  st.add(init_out, (size_t)npix * 10 * sizeof(float), true);
  st.add(pol_out, pol_out ? (size_t)npix * sizeof(float) : 0, true);
  if ((rc = st.prepare(h, s))) return rc;
  if (launch_weak_field((const float*)st.bufs[0].dev, npix, nullptr, (const float*)st.bufs[1].dev, nfilt,
                        (const float*)st.bufs[2].dev, nlam, line_constants(line), 0, 0.0f,
                        h->geom, (float*)st.bufs[3].dev, (float*)st.bufs[4].dev,
                        s) != cudaSuccess)
    return VFISV_E_CUDA;
  return st.finish(s);
}

int vfisv_restart_models(vfisv_handle* h, const float* models, int64_t n, int64_t pixel0,
                         int32_t k, uint32_t free_mask, uint64_t seed, float* models_out,
                         void* stream) {
  if (!h || !models || !models_out || (free_mask & ~0x1FFu)) return VFISV_E_ARG;
  if (n < 0 || pixel0 < 0 || pixel0 + n > (1ll << 40) || k < 1 || k >= (1 << 20))
    return VFISV_E_SIZE;
  if (n == 0) return VFISV_OK;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Staging st;
  st.add(models, (size_t)n * 10 * sizeof(float), false);
  st.add(models_out, (size_t)n * 10 * sizeof(float), true);
  int rc = st.prepare(h, s);
  if (rc) return rc;
  if (launch_restart_perturb((const float*)st.bufs[0].dev, n, pixel0, k, free_mask, seed,
                             (float*)st.bufs[1].dev, s) != cudaSuccess)
    return VFISV_E_CUDA;
  return st.finish(s);
}

int vfisv_limb_weights(vfisv_handle* h, const float* obs, const float* mu, int64_t npix,
                       int32_t nfilt, float ic0, const float* sigma4, float* weights_out,
                       void* stream) {
  if (!h || !obs || !mu || !sigma4 || !weights_out || !(ic0 > 0)) return VFISV_E_ARG;
  for (int i = 0; i < 4; ++i)
    if (!(sigma4[i] > 0)) return VFISV_E_ARG;
  if (npix < 0 || nfilt < 1 || nfilt > 64) return VFISV_E_SIZE;
  if (npix == 0) return VFISV_OK;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Staging st;
  st.add(obs, (size_t)npix * 4 * nfilt * sizeof(float), false);
  st.add(mu, (size_t)npix * sizeof(float), false);
  st.add(weights_out, (size_t)npix * 4 * nfilt * sizeof(float), true);
  int rc = st.prepare(h, s);
  if (rc) return rc;
  if (launch_limb_weights((const float*)st.bufs[0].dev, (const float*)st.bufs[1].dev, npix, nfilt,
                          ic0, sigma4, (float*)st.bufs[2].dev, s) != cudaSuccess)
    return VFISV_E_CUDA;
  return st.finish(s);
}

int vfisv_check(vfisv_handle* h, void* stream) {
  if (!h) return VFISV_E_ARG;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) return VFISV_E_CUDA;
  if (cudaGetLastError() != cudaSuccess) return VFISV_E_CUDA;
  // error words: the inversion workspace and the network workspace
  int bad = 0;
  for (void* w : {h->ws, h->nnws}) {
    if (!w) continue;
    int e = 0;
    if (cudaMemcpy(&e, w, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return VFISV_E_CUDA;
    if (e) {
      cudaMemset(w, 0, sizeof(int));
      bad = 1;
    }
  }
  return bad ? VFISV_E_DEVICE : VFISV_OK;
}

int vfisv_synth(vfisv_handle* h, const float* params, int64_t npix, const float* filters,
                int32_t nfilt, const float* wl_mA, int32_t nlam, const vfisv_line* line,
                float* stokes, void* stream) {
  if (!h || !params || !filters || !wl_mA || !stokes || !line_ok(line)) return VFISV_E_ARG;
  if (npix < 0 || nfilt < 1 || nlam < 1 || nlam > 4096) return VFISV_E_SIZE;
  if (nfilt > 8 && !wide_supported(nfilt, nlam)) return VFISV_E_UNSUPPORTED;
  if (npix == 0) return VFISV_OK;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  WsLayout L = layout(nfilt, nlam, 0, false);
  if (h->ws_bytes < L.total) {
    int rc = grow(&h->ws, &h->ws_bytes, L.total);
    if (rc) return rc;
    if (cudaMemsetAsync(h->ws, 0, 64, s) != cudaSuccess) return VFISV_E_CUDA;
  }
  Staging st;
  st.add(params, (size_t)npix * 10 * sizeof(float), false);
  st.add(filters, (size_t)nfilt * nlam * sizeof(float), false);
  st.add(wl_mA, (size_t)nlam * sizeof(float), false);
  st.add(stokes, (size_t)npix * 4 * nfilt * sizeof(float), true);
  int rc = st.prepare(h, s);
  if (rc) return rc;
  char* ws = (char*)h->ws;
  float* table = (float*)(ws + L.table);
  if (nfilt > 8) {  // many narrow instrument profiles: one pixel per warp
    int* err = (int*)(ws + L.err);
    if (launch_wide_pack((const float*)st.bufs[1].dev, nfilt, (const float*)st.bufs[2].dev, nlam,
                         table, err, s) != cudaSuccess ||
        launch_wide_synth((const float*)st.bufs[0].dev, npix, table, nfilt, nlam,
                          (float*)st.bufs[3].dev, err, h->W, line_constants(line), s) !=
            cudaSuccess)
      return VFISV_E_CUDA;
    return st.finish(s);
  }
  if (launch_pack_table((const float*)st.bufs[1].dev, nfilt, (const float*)st.bufs[2].dev,
                        nlam, table, s) != cudaSuccess)
    return VFISV_E_CUDA;
  SynthArgs a;
  a.params = (const float*)st.bufs[0].dev;
  a.npix = npix;
  a.table = table;
  a.nlam = nlam;
  a.stokes = (float*)st.bufs[3].dev;
  a.err = (int*)(ws + L.err);
  a.W = h->W;
  a.lk = line_constants(line);
  if (launch_synth(a, nfilt, s) != cudaSuccess) return VFISV_E_CUDA;
  return st.finish(s);
}

int vfisv_invert(vfisv_handle* h, const float* obs, const float* weights,
                 int32_t weights_per_pixel, const float* filters, int32_t nfilt,
                 const float* wl_mA, int32_t nlam, const vfisv_line* line, const float* init,
                 const vfisv_config* cfg, int64_t npix, float* params_out, float* chi2_out,
                 int32_t* iters_out, int32_t* status_out, float* cov_out, void* stream) {
  int rc = check_invert_args(h, obs, weights, filters, nfilt, wl_mA, nlam, line, cfg, npix,
                             params_out, chi2_out, iters_out, status_out);
  if (rc || npix == 0) return rc;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int nobs = 4 * nfilt;
  if (pipeline_host(h, obs, npix, cfg->restarts == 0)) {
    // shared inputs once, the per-pixel rows through the pipeline
    Staging sh;
    sh.add(filters, (size_t)nfilt * nlam * sizeof(float), false);
    sh.add(wl_mA, (size_t)nlam * sizeof(float), false);
    sh.add(weights_per_pixel ? nullptr : weights, (size_t)nobs * sizeof(float), false);
    if ((rc = sh.prepare(h, s))) return rc;
    const float* fd = (const float*)sh.bufs[0].dev;
    const float* wd = (const float*)sh.bufs[1].dev;
    const float* wsh = (const float*)sh.bufs[2].dev;
    RowArg a[] = {{obs, nobs * sizeof(float), false},
                  {weights_per_pixel ? weights : nullptr, nobs * sizeof(float), false},
                  {init, 10 * sizeof(float), false},
                  {params_out, 10 * sizeof(float), true},
                  {chi2_out, sizeof(float), true},
                  {iters_out, sizeof(int32_t), true},
                  {status_out, sizeof(int32_t), true},
                  {cov_out, 100 * sizeof(float), true}};
    return pipeline_rows(h, s, npix, a, 8, [&](int64_t n, void** d) {
      // every pointer is on the device: the call runs in place, without syncing
      return vfisv_invert(h, (const float*)d[0], weights_per_pixel ? (const float*)d[1] : wsh,
                          weights_per_pixel, fd, nfilt, wd, nlam, line, (const float*)d[2], cfg,
                          n, (float*)d[3], (float*)d[4], (int32_t*)d[5], (int32_t*)d[6],
                          (float*)d[7], s);
    });
  }
  Staging st;
  st.add(obs, (size_t)npix * nobs * sizeof(float), false);
  st.add(weights, (size_t)(weights_per_pixel ? npix : 1) * nobs * sizeof(float), false);
  st.add(filters, (size_t)nfilt * nlam * sizeof(float), false);
  st.add(wl_mA, (size_t)nlam * sizeof(float), false);
  st.add(init, init ? (size_t)npix * 10 * sizeof(float) : 0, false);
  st.add(params_out, (size_t)npix * 10 * sizeof(float), true);
  st.add(chi2_out, (size_t)npix * sizeof(float), true);
  st.add(iters_out, (size_t)npix * sizeof(int32_t), true);
  st.add(status_out, (size_t)npix * sizeof(int32_t), true);
  st.add(cov_out, cov_out ? (size_t)npix * 100 * sizeof(float) : 0, true);
  if ((rc = st.prepare(h, s))) return rc;
  DevInvert d;
  d.obs = (const float*)st.bufs[0].dev;
  d.w = (const float*)st.bufs[1].dev;
  d.w_stride = weights_per_pixel ? nobs : 0;
  d.filters = (const float*)st.bufs[2].dev;
  d.wl = (const float*)st.bufs[3].dev;
  d.init = (const float*)st.bufs[4].dev;
  d.params = (float*)st.bufs[5].dev;
  d.chi2 = (float*)st.bufs[6].dev;
  d.iters = (int32_t*)st.bufs[7].dev;
  d.status = (int32_t*)st.bufs[8].dev;
  d.cov = (float*)st.bufs[9].dev;
  if ((rc = invert_device(h, d, nfilt, nlam, line, cfg, npix, nullptr, s))) return rc;
  return st.finish(s);
}

int vfisv_nn_init(vfisv_handle* h, float* blob, const float* obs, const float* params,
                  int64_t n, uint64_t seed, void* stream) {
  if (!h || !blob || !obs || !params) return VFISV_E_ARG;
  if (n < 1) return VFISV_E_SIZE;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Staging st;
  st.add(blob, nn::NBLOB * sizeof(float), true);
  st.add(obs, (size_t)n * nn::IN * sizeof(float), false);
  st.add(params, (size_t)n * 10 * sizeof(float), false);
  int rc = st.prepare(h, s);
  if (rc) return rc;
  if ((rc = grow(&h->nnws, &h->nnws_bytes, nn::workspace_bytes(512)))) return rc;
  if (nn::nn_init(h->nnws, (float*)st.bufs[0].dev, (const float*)st.bufs[1].dev,
                  (const float*)st.bufs[2].dev, n, seed, s) != cudaSuccess)
    return VFISV_E_CUDA;
  return st.finish(s);
}

int vfisv_nn_train(vfisv_handle* h, float* blob, const float* obs, const float* params,
                   int64_t n, int32_t batch, int32_t epochs, float lr0, uint64_t seed,
                   float* loss_hist, void* stream) {
  if (!h || !blob || !obs || !params || !(lr0 > 0) || epochs < 0) return VFISV_E_ARG;
  if (batch < 512 || batch % 512 != 0 || n < batch || n >= (1ll << 31)) return VFISV_E_SIZE;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t steps = (n / batch) * epochs;
  Staging st;
  st.add(blob, nn::NBLOB * sizeof(float), false);
  st.add(obs, (size_t)n * nn::IN * sizeof(float), false);
  st.add(params, (size_t)n * 10 * sizeof(float), false);
  st.add(loss_hist, loss_hist ? (size_t)steps * sizeof(float) : 0, true);
  int rc = st.prepare(h, s);
  if (rc) return rc;
  // the blob is updated in place: a host blob is copied back after training
  st.bufs[0].out = true;
  if ((rc = grow(&h->nnws, &h->nnws_bytes, nn::workspace_bytes(batch)))) return rc;
  if (nn::nn_train(h->nnws, (float*)st.bufs[0].dev, (const float*)st.bufs[1].dev,
                   (const float*)st.bufs[2].dev, n, batch, epochs, lr0, seed,
                   (float*)st.bufs[3].dev, s) != cudaSuccess)
    return VFISV_E_CUDA;
  return st.finish(s);
}

int vfisv_nn_grad(vfisv_handle* h, const float* blob, const float* obs, const float* params,
                  int64_t n, float* grad_out, float* loss_out, void* stream) {
  if (!h || !blob || !obs || !params || !grad_out || !loss_out) return VFISV_E_ARG;
  if (n < 1 || n > (1ll << 20)) return VFISV_E_SIZE;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Staging st;
  st.add(blob, nn::NBLOB * sizeof(float), false);
  st.add(obs, (size_t)n * nn::IN * sizeof(float), false);
  st.add(params, (size_t)n * 10 * sizeof(float), false);
  st.add(grad_out, nn::NTRAIN * sizeof(float), true);
  st.add(loss_out, sizeof(float), true);
  int rc = st.prepare(h, s);
  if (rc) return rc;
  if ((rc = grow(&h->nnws, &h->nnws_bytes, nn::workspace_bytes(nn::padded_rows(n))))) return rc;
  if (nn::nn_grad(h->nnws, (const float*)st.bufs[0].dev, (const float*)st.bufs[1].dev,
                  (const float*)st.bufs[2].dev, n, (float*)st.bufs[3].dev,
                  (float*)st.bufs[4].dev, s) != cudaSuccess)
    return VFISV_E_CUDA;
  return st.finish(s);
}

int vfisv_nn_infer(vfisv_handle* h, const float* blob, const float* obs, int64_t npix,
                   const vfisv_line* line, float* init_out, float* conf_out, float* raw_out,
                   void* stream) {
  if (!h || !blob || !obs || !init_out || !line_ok(line)) return VFISV_E_ARG;
  if (npix < 0) return VFISV_E_SIZE;
  if (npix == 0) return VFISV_OK;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Staging st;
  st.add(blob, nn::NBLOB * sizeof(float), false);
  st.add(obs, (size_t)npix * nn::IN * sizeof(float), false);
  st.add(init_out, (size_t)npix * 10 * sizeof(float), true);
  st.add(conf_out, conf_out ? (size_t)npix * sizeof(float) : 0, true);
  st.add(raw_out, raw_out ? (size_t)npix * nn::OUT * sizeof(float) : 0, true);
  int rc = st.prepare(h, s);
  if (rc) return rc;
  if ((rc = grow(&h->nnws, &h->nnws_bytes, nn::infer_workspace_bytes()))) return rc;
  if (nn::nn_infer(h->nnws, (const float*)st.bufs[0].dev,
                   (const float*)st.bufs[1].dev, npix, (float)line->mu,
                   (float*)st.bufs[2].dev, (float*)st.bufs[3].dev, (float*)st.bufs[4].dev,
                   s) != cudaSuccess)
    return VFISV_E_CUDA;
  return st.finish(s);
}

int vfisv_invert_batch(vfisv_handle* h, const float* obs, const float* weights,
                       const int64_t* map_off, int32_t nmaps, const float* filters,
                       int32_t nfilt, const float* wl_mA, int32_t nlam, const vfisv_line* line,
                       const float* init, const vfisv_config* cfg, float* params_out,
                       float* chi2_out, int32_t* iters_out, int32_t* status_out, float* cov_out,
                       float* latency_ms, void* stream) {
  if (!map_off || nmaps < 1) return VFISV_E_ARG;
  if (map_off[0] != 0) return VFISV_E_ARG;
  for (int m = 0; m < nmaps; ++m)
    if (map_off[m + 1] < map_off[m]) return VFISV_E_ARG;
  const int64_t npix = map_off[nmaps];
  int rc = check_invert_args(h, obs, weights, filters, nfilt, wl_mA, nlam, line, cfg, npix,
                             params_out, chi2_out, iters_out, status_out);
  if (rc) return rc;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int nobs = 4 * nfilt;
  // device: offsets [nmaps+1], completion counters [nmaps], stamps [nmaps], start stamp
  const size_t b_off = up((size_t)(nmaps + 1) * 8), b_cnt = up((size_t)nmaps * 8);
  if ((rc = grow(&h->mapws, &h->mapws_bytes, b_off + 2 * b_cnt + 256))) return rc;
  const size_t hbytes = (size_t)(nmaps + 1) * 8;
  if (h->mapoff_host_bytes < hbytes) {
    if (t_capturing) return VFISV_E_CAPTURE;
    if (h->mapoff_host) cudaFreeHost(h->mapoff_host);
    h->mapoff_host = nullptr;
    h->mapoff_host_bytes = 0;
    if (cudaMallocHost((void**)&h->mapoff_host, hbytes) != cudaSuccess) return VFISV_E_NOMEM;
    h->mapoff_host_bytes = hbytes;
  }
  // the pinned copy is read by the copy below (and by every replay of a
  // captured graph), so the caller's array need not outlive the call; an
  // earlier call's copy from it must be complete before it is rewritten
  if (!t_capturing && cudaStreamSynchronize(s) != cudaSuccess) return VFISV_E_CUDA;
  memcpy(h->mapoff_host, map_off, hbytes);
  char* mw = (char*)h->mapws;
  int64_t* off_d = (int64_t*)mw;
  unsigned long long* done = (unsigned long long*)(mw + b_off);
  unsigned long long* tdone = (unsigned long long*)(mw + b_off + b_cnt);
  unsigned long long* t0 = (unsigned long long*)(mw + b_off + 2 * b_cnt);
  if (cudaMemcpyAsync(off_d, h->mapoff_host, hbytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(done, 0, b_cnt, s) != cudaSuccess ||
      cudaMemsetAsync(tdone, 0, b_cnt, s) != cudaSuccess)
    return VFISV_E_CUDA;
  if (npix == 0) {  // every map empty: latencies 0
    if (!latency_ms) return VFISV_OK;
    if (is_device_ptr(latency_ms))
      return cudaMemsetAsync(latency_ms, 0, (size_t)nmaps * sizeof(float), s) == cudaSuccess
                 ? VFISV_OK
                 : VFISV_E_CUDA;
    memset(latency_ms, 0, (size_t)nmaps * sizeof(float));
    return VFISV_OK;
  }
  Staging st;
  st.add(obs, (size_t)npix * nobs * sizeof(float), false);
  st.add(weights, (size_t)nmaps * nobs * sizeof(float), false);
  st.add(filters, (size_t)nfilt * nlam * sizeof(float), false);
  st.add(wl_mA, (size_t)nlam * sizeof(float), false);
  st.add(init, init ? (size_t)npix * 10 * sizeof(float) : 0, false);
  st.add(params_out, (size_t)npix * 10 * sizeof(float), true);
  st.add(chi2_out, (size_t)npix * sizeof(float), true);
  st.add(iters_out, (size_t)npix * sizeof(int32_t), true);
  st.add(status_out, (size_t)npix * sizeof(int32_t), true);
  st.add(cov_out, cov_out ? (size_t)npix * 100 * sizeof(float) : 0, true);
  st.add(latency_ms, latency_ms ? (size_t)nmaps * sizeof(float) : 0, true);
  if ((rc = st.prepare(h, s))) return rc;
  if (launch_stamp(t0, s) != cudaSuccess) return VFISV_E_CUDA;
  DevInvert d;
  d.obs = (const float*)st.bufs[0].dev;
  d.w = (const float*)st.bufs[1].dev;
  d.w_stride = 0;
  d.filters = (const float*)st.bufs[2].dev;
  d.wl = (const float*)st.bufs[3].dev;
  d.init = (const float*)st.bufs[4].dev;
  d.params = (float*)st.bufs[5].dev;
  d.chi2 = (float*)st.bufs[6].dev;
  d.iters = (int32_t*)st.bufs[7].dev;
  d.status = (int32_t*)st.bufs[8].dev;
  d.cov = (float*)st.bufs[9].dev;
  d.map_off = off_d;
  d.nmaps = nmaps;
  d.map_done = done;
  d.map_t = tdone;
  if ((rc = invert_device(h, d, nfilt, nlam, line, cfg, npix, nullptr, s))) return rc;
  if (latency_ms && launch_map_latency(tdone, t0, nmaps, (float*)st.bufs[10].dev, s) !=
                        cudaSuccess)
    return VFISV_E_CUDA;
  return st.finish(s);
}

int vfisv_invert_nn(vfisv_handle* h, const float* blob, const float* obs, const float* weights,
                    int32_t weights_per_pixel, const float* filters, int32_t nfilt,
                    const float* wl_mA, int32_t nlam, const vfisv_line* line,
                    const vfisv_config* cfg_nn, const vfisv_config* cfg_plain,
                    double chi2_flag, int32_t flag_unconverged, double conf_route,
                    int64_t npix, float* params_out, float* chi2_out,
                    int32_t* iters_out, int32_t* status_out, float* cov_out,
                    int32_t* flagged_out, void* stream) {
  if (!blob || !cfg_plain || isnan(conf_route)) return VFISV_E_ARG;
  int rc = check_invert_args(h, obs, weights, filters, nfilt, wl_mA, nlam, line, cfg_nn, npix,
                             params_out, chi2_out, iters_out, status_out);
  if (rc) return rc;
  if ((rc = check_config(cfg_plain, nfilt))) return rc;
  if (nfilt != nn::IN / 4) return VFISV_E_UNSUPPORTED;
  if (npix == 0) return VFISV_OK;
  if (set_device(h)) return VFISV_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int nobs = 4 * nfilt;
  if (pipeline_host(h, obs, npix, cfg_nn->restarts == 0 && cfg_plain->restarts == 0)) {
    Staging sh;
    sh.add(filters, (size_t)nfilt * nlam * sizeof(float), false);
    sh.add(wl_mA, (size_t)nlam * sizeof(float), false);
    sh.add(blob, nn::NBLOB * sizeof(float), false);
    sh.add(weights_per_pixel ? nullptr : weights, (size_t)nobs * sizeof(float), false);
    if ((rc = sh.prepare(h, s))) return rc;
    const float* fd = (const float*)sh.bufs[0].dev;
    const float* wd = (const float*)sh.bufs[1].dev;
    const float* bd = (const float*)sh.bufs[2].dev;
    const float* wsh = (const float*)sh.bufs[3].dev;
    RowArg a[] = {{obs, nobs * sizeof(float), false},
                  {weights_per_pixel ? weights : nullptr, nobs * sizeof(float), false},
                  {params_out, 10 * sizeof(float), true},
                  {chi2_out, sizeof(float), true},
                  {iters_out, sizeof(int32_t), true},
                  {status_out, sizeof(int32_t), true},
                  {cov_out, 100 * sizeof(float), true},
                  {flagged_out, sizeof(int32_t), true}};
    return pipeline_rows(h, s, npix, a, 8, [&](int64_t n, void** d) {
      // every pointer is on the device: the call runs in place, without syncing
      return vfisv_invert_nn(h, bd, (const float*)d[0],
                             weights_per_pixel ? (const float*)d[1] : wsh, weights_per_pixel, fd,
                             nfilt, wd, nlam, line, cfg_nn, cfg_plain, chi2_flag,
                             flag_unconverged, conf_route, n, (float*)d[2], (float*)d[3],
                             (int32_t*)d[4],
                             (int32_t*)d[5], (float*)d[6], (int32_t*)d[7], s);
    });
  }
  Staging st;
  st.add(obs, (size_t)npix * nobs * sizeof(float), false);
  st.add(weights, (size_t)(weights_per_pixel ? npix : 1) * nobs * sizeof(float), false);
  st.add(filters, (size_t)nfilt * nlam * sizeof(float), false);
  st.add(wl_mA, (size_t)nlam * sizeof(float), false);
  st.add(blob, nn::NBLOB * sizeof(float), false);
  st.add(params_out, (size_t)npix * 10 * sizeof(float), true);
  st.add(chi2_out, (size_t)npix * sizeof(float), true);
  st.add(iters_out, (size_t)npix * sizeof(int32_t), true);
  st.add(status_out, (size_t)npix * sizeof(int32_t), true);
  st.add(cov_out, cov_out ? (size_t)npix * 100 * sizeof(float) : 0, true);
  st.add(flagged_out, flagged_out ? (size_t)npix * sizeof(int32_t) : 0, true);
  if ((rc = st.prepare(h, s))) return rc;
  const float* o = (const float*)st.bufs[0].dev;
  const float* w = (const float*)st.bufs[1].dev;
  const int64_t wstride = weights_per_pixel ? nobs : 0;
  // workspace: guesses, index, count, gathered obs/weights, second-run outputs
  const bool cov = cov_out != nullptr;
  size_t off = 0;
  auto place = [&](size_t bytes) {
    const size_t at = off;
    off += up(bytes);
    return at;
  };
  const bool route = isfinite(conf_route) != 0;
  const size_t o_init = place((size_t)npix * 10 * 4), o_cnt = place(8),
               o_conf = route ? place((size_t)npix * 4) : 0, o_rcnt = route ? place(8) : 0,
               o_idx = place((size_t)npix * 8), o_obs = place((size_t)npix * nobs * 4),
               o_w = weights_per_pixel ? place((size_t)npix * nobs * 4) : 0,
               o_p = place((size_t)npix * 10 * 4), o_c = place((size_t)npix * 4),
               o_i = place((size_t)npix * 4), o_s = place((size_t)npix * 4),
               o_v = cov ? place((size_t)npix * 100 * 4) : 0;
  if ((rc = grow(&h->mixws, &h->mixws_bytes, off))) return rc;
  if ((rc = grow(&h->nnws, &h->nnws_bytes, nn::infer_workspace_bytes()))) return rc;
  char* mw = (char*)h->mixws;
  float* init = (float*)(mw + o_init);
  float* conf = route ? (float*)(mw + o_conf) : nullptr;
  if (nn::nn_infer(h->nnws, (const float*)st.bufs[4].dev, o, npix, (float)line->mu,
                   init, conf, nullptr, s) != cudaSuccess)
    return VFISV_E_CUDA;
  if (cfg_nn->wfa_pol > 0.0) {
    // the paper's combination (Sec. 5): weak-field B, gamma below the
    // polarisation threshold, the wing azimuth everywhere
    if ((rc = grow(&h->geom, &h->geom_bytes, filter_geom_bytes()))) return rc;
    if (launch_weak_field(o, npix, nullptr, (const float*)st.bufs[2].dev, nfilt,
                          (const float*)st.bufs[3].dev, nlam, line_constants(line), 1,
                          (float)cfg_nn->wfa_pol, h->geom, init, nullptr, s) != cudaSuccess)
      return VFISV_E_CUDA;
  }
  DevInvert d;
  d.obs = o;
  d.w = w;
  d.w_stride = wstride;
  d.filters = (const float*)st.bufs[2].dev;
  d.wl = (const float*)st.bufs[3].dev;
  d.init = init;
  d.params = (float*)st.bufs[5].dev;
  d.chi2 = (float*)st.bufs[6].dev;
  d.iters = (int32_t*)st.bufs[7].dev;
  d.status = (int32_t*)st.bufs[8].dev;
  d.cov = (float*)st.bufs[9].dev;
  // with the same solve settings in both runs the covariance is computed once,
  // over the merged rows, from the J^T W J each run parks there
  const bool one_cov = cov && cfg_nn->free_mask == cfg_plain->free_mask &&
                       cfg_nn->fast_solve == cfg_plain->fast_solve;
  d.park_cov = one_cov;
  int64_t* cnt = (int64_t*)(mw + o_cnt);
  int64_t* idx = (int64_t*)(mw + o_idx);
  const int64_t* n_first = nullptr;
  if (route) {
    // the pixels the network is confident about run LM from its guess;
    // the others go straight to the plain run (their list reuses idx,
    // which the flag step overwrites only after the first run)
    int64_t* rcnt = (int64_t*)(mw + o_rcnt);
    if (nn::route_by_confidence(conf, npix, (float)conf_route, init, idx, rcnt, d.params, d.chi2,
                                d.iters, d.status, s) != cudaSuccess)
      return VFISV_E_CUDA;
    d.pix_list = idx;
    n_first = rcnt;
  }
  if ((rc = invert_device(h, d, nfilt, nlam, line, cfg_nn, npix, n_first, s))) return rc;
  float* og = (float*)(mw + o_obs);
  float* wg = weights_per_pixel ? (float*)(mw + o_w) : nullptr;
  if (nn::flag_and_gather(d.status, d.chi2, npix, (float)chi2_flag, flag_unconverged != 0, o, w,
                          wstride, nobs, cnt, idx, og, wg, (int32_t*)st.bufs[10].dev,
                          s) != cudaSuccess)
    return VFISV_E_CUDA;
  DevInvert d2;
  d2.obs = og;
  d2.w = weights_per_pixel ? wg : w;
  d2.w_stride = wstride;
  d2.filters = d.filters;
  d2.wl = d.wl;
  d2.init = nullptr;
  d2.params = (float*)(mw + o_p);
  d2.chi2 = (float*)(mw + o_c);
  d2.iters = (int32_t*)(mw + o_i);
  d2.status = (int32_t*)(mw + o_s);
  d2.cov = cov ? (float*)(mw + o_v) : nullptr;
  d2.park_cov = one_cov;
  if ((rc = invert_device(h, d2, nfilt, nlam, line, cfg_plain, npix, cnt, s))) return rc;
  if (nn::merge_plain(cnt, idx, npix, d2.params, d2.chi2, d2.iters, d2.status, d2.cov, d.params,
                      d.chi2, d.iters, d.status, d.cov, s) != cudaSuccess)
    return VFISV_E_CUDA;
  if (one_cov && launch_covariance(d.cov, d.status, npix, nullptr, cfg_plain->free_mask,
                                   cfg_plain->fast_solve, s) != cudaSuccess)
    return VFISV_E_CUDA;
  return st.finish(s);
}

}  // extern "C"
