// Initial-guess network (Sec. 5): a 24-256-256-256-11 multilayer perceptron
// with GELU activations, trained and evaluated by hand-written BF16
// tensor-core kernels with FP32 accumulation: the training products run on
// tcgen05 (nn_tc.cu), inference in one fused tcgen05 kernel (mlp_tc.cu).
// This file holds the rest of training: features and targets, the loss and
// its gradient, bias gradients, the split-K reduction, Adam, weight packing,
// initialisation and the standardisation statistics, and the host driver.
//
// Parameter blob (float32, see vfisv.h): W0[24][256] b0[256] W1[256][256]
// b1[256] W2[256][256] b2[256] W3[256][11] b3[11] in_mean[24] in_std[24]
// out_mean[10] out_std[10]; weights are [fan_in][fan_out] (y = x W + b).
#include <cuda_bf16.h>
#include <math.h>

#include <vector>

#include "common.cuh"
#include "nn.cuh"
#include "nn_device.cuh"
#include "nn_tc.cuh"

namespace vfisv {
namespace nn {

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------------------
// Features, targets, decoding (the network's view of a pixel).
//
// Features: f_j = (obs_j / Ic - in_mean_j) / in_std_j, Ic = max(largest I
// sample, 1e-30).  Targets (standardised with out_mean/out_std):
// [B, cos gamma, sin 2psi, cos 2psi, ln eta0, dlambdaD, a, v, S0/Ic, S1/Ic].

// mult < n, offset + m < 2n and n < 2^31 keep the product inside 64 bits.
__device__ __forceinline__ int64_t sample_of(int64_t m, const Perm& p) {
  return (int64_t)((p.mult * (uint64_t)(p.offset + m) + p.add) % (uint64_t)p.n);
}

// Padded widths of the training operands: the input features (24) fill one
// 64-column K-chunk; their transposed copy (a weight-gradient operand of N =
// 32) has 32 rows; the outputs (11) are a 16-column tile, their gradient a
// 64-column K-chunk.
constexpr int XK = 64, XT = 32, YN = 16, DYK = 64;

__device__ __forceinline__ void put_bf16(uint8_t* base, size_t off, float v) {
  *reinterpret_cast<bf16*>(base + off) = __float2bfloat16(v);
}

// Features of row m (sample perm(m)) into X0 = TL(mpad, 64) and its
// transpose X0T = TL(32, mpad); rows past `rows` and the padding are zero.
__global__ void features_kernel(const float* __restrict__ obs, int64_t rows, int64_t mpad,
                                Perm perm, const float* __restrict__ blob,
                                uint8_t* __restrict__ X, uint8_t* __restrict__ XTr,
                                float* __restrict__ ic_out) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= mpad) return;
  float f[XT];
#pragma unroll
  for (int j = 0; j < XT; ++j) f[j] = 0.0f;
  float ic = 1.0f;
  if (m < rows) {
    const int64_t s = sample_of(m, perm);
    const float* o = obs + s * IN;
    ic = ic_of(o);
    const float inv = 1.0f / ic;
#pragma unroll
    for (int j = 0; j < IN; ++j) f[j] = (o[j] * inv - blob[OFF_INM + j]) / blob[OFF_INS + j];
  }
  for (int j = 0; j < XK; j += 8) {
    uint4 pk = make_uint4(0u, 0u, 0u, 0u);
    if (j < XT) {
      __nv_bfloat162 t0 = __floats2bfloat162_rn(f[j], f[j + 1]);
      __nv_bfloat162 t1 = __floats2bfloat162_rn(f[j + 2], f[j + 3]);
      __nv_bfloat162 t2 = __floats2bfloat162_rn(f[j + 4], f[j + 5]);
      __nv_bfloat162 t3 = __floats2bfloat162_rn(f[j + 6], f[j + 7]);
      pk = make_uint4(*reinterpret_cast<uint32_t*>(&t0), *reinterpret_cast<uint32_t*>(&t1),
                      *reinterpret_cast<uint32_t*>(&t2), *reinterpret_cast<uint32_t*>(&t3));
    }
    *reinterpret_cast<uint4*>(X + tl_off(m, j, mpad)) = pk;
  }
#pragma unroll
  for (int j = 0; j < XT; ++j) put_bf16(XTr, tl_off(j, m, XT), f[j]);
  ic_out[m] = ic;
}

__device__ __forceinline__ void targets(const float* p, float ic, float (&t)[OUT - 1]) {
  const float g = p[1] * 0.017453292519943295f, ps = p[2] * 0.034906585039886591f;
  t[0] = p[0];
  t[1] = cosf(g);
  t[2] = sinf(ps);
  t[3] = cosf(ps);
  t[4] = logf(p[3]);
  t[5] = p[4];
  t[6] = p[5];
  t[7] = p[6];
  t[8] = p[7] / ic;
  t[9] = p[8] / ic;
}

// Loss of Sec. 5's regression plus the confidence output, and dL/dy: the
// outputs Y [mpad][16] (FP32), the gradient into dY = TL(mpad, 64) and
// dYT = TL(16, mpad) (BF16; zero on padding rows and columns).
__global__ void loss_kernel(const float* __restrict__ Y, int64_t rows, int64_t mpad, Perm perm,
                            const float* __restrict__ params, const float* __restrict__ ic,
                            const float* __restrict__ blob, uint8_t* __restrict__ dY,
                            uint8_t* __restrict__ dYT, float* __restrict__ partial) {
  __shared__ float red[256];
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (m < mpad) {
    float d[YN];
#pragma unroll
    for (int o = 0; o < YN; ++o) d[o] = 0.0f;
    if (m < rows) {
      const int64_t s = sample_of(m, perm);
      float t[OUT - 1];
      targets(params + s * 10, ic[m], t);
      const float* y = Y + m * YN;
      const float invn = 1.0f / (float)rows;
      float e[OUT - 1], mse = 0.0f;
#pragma unroll
      for (int o = 0; o < OUT - 1; ++o) {
        const float ts = (t[o] - blob[OFF_OUTM + o]) / blob[OFF_OUTS + o];
        e[o] = y[o] - ts;
        mse = fmaf(e[o], e[o], mse);
      }
      const float c = logf(mse / (OUT - 1) + 1e-4f);
      const float ec = y[OUT - 1] - c;
      l = mse * invn / (OUT - 1) + ec * ec * invn;
#pragma unroll
      for (int o = 0; o < OUT - 1; ++o) d[o] = 2.0f * e[o] * invn / (OUT - 1);
      d[OUT - 1] = 2.0f * ec * invn;
    }
    for (int j = 0; j < DYK; j += 8) {
      uint4 pk = make_uint4(0u, 0u, 0u, 0u);
      if (j < YN) {
        __nv_bfloat162 t0 = __floats2bfloat162_rn(d[j], d[j + 1]);
        __nv_bfloat162 t1 = __floats2bfloat162_rn(d[j + 2], d[j + 3]);
        __nv_bfloat162 t2 = __floats2bfloat162_rn(d[j + 4], d[j + 5]);
        __nv_bfloat162 t3 = __floats2bfloat162_rn(d[j + 6], d[j + 7]);
        pk = make_uint4(*reinterpret_cast<uint32_t*>(&t0), *reinterpret_cast<uint32_t*>(&t1),
                        *reinterpret_cast<uint32_t*>(&t2), *reinterpret_cast<uint32_t*>(&t3));
      }
      *reinterpret_cast<uint4*>(dY + tl_off(m, j, mpad)) = pk;
    }
#pragma unroll
    for (int o = 0; o < YN; ++o) put_bf16(dYT, tl_off(o, m, YN), d[o]);
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Bias gradients: row sums of a transposed gradient GT = TL(N, M) (the sum
// over the batch of each output's gradient) over batch chunks of `chunk`
// columns (a multiple of 64): partial[s][N].  One warp per 8-row group and
// chunk: a 64-column block of the group is 1024 contiguous bytes, 64 segments
// of 16 bytes, segment j holding row j % 8; lane l loads segments l and l + 32
// (both row l % 8), and lanes of one row combine by xor-shuffles in a fixed
// order.
__global__ void rowsum_kernel(const uint8_t* __restrict__ GT, int N, int64_t M, int64_t chunk,
                              float* __restrict__ partial) {
  const int grp = blockIdx.x, s = blockIdx.y, lane = threadIdx.x;
  const int64_t m0 = (int64_t)s * chunk, m1 = (m0 + chunk < M) ? m0 + chunk : M;
  float acc = 0.0f;
  for (int64_t c = m0; c < m1; c += 64) {
    const uint8_t* blk = GT + tl_off((int64_t)grp * 8, (int)c, N);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint4 q = *reinterpret_cast<const uint4*>(blk + 16 * (lane + 32 * h));
      const __nv_bfloat162* e = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 f = __bfloat1622float2(e[k]);
        acc += f.x + f.y;
      }
    }
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 8);
  acc += __shfl_xor_sync(0xffffffffu, acc, 16);
  if (lane < 8) partial[(size_t)s * N + grp * 8 + lane] = acc;
}

// Sum split-K partials into the gradient blob (fixed order: deterministic).
struct GradLayer {
  const float* wpart;  // [splits][GM][GN]
  const float* bpart;  // [splits][Np]
  int GM, GN;          // GEMM output shape (transposed: [Np][Kp], else [Kp][Np])
  int K, N;            // logical fan_in, fan_out
  int transposed;
  int wsplits, bsplits;
  size_t offW, offB;
};
struct GradArgs {
  GradLayer L[4];
  float* grad;
  const float* loss_partial;
  int nloss;
  float* loss_out;
};

__global__ void reduce_grad_kernel(GradArgs a) {
  const int l = blockIdx.y;
  const GradLayer& G = a.L[l];
  const int total = G.K * G.N + G.N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    float s = 0.0f;
    if (i < G.K * G.N) {
      const int k = i / G.N, n = i % G.N;
      const size_t e = G.transposed ? (size_t)n * G.GN + k : (size_t)k * G.GN + n;
      for (int q = 0; q < G.wsplits; ++q) s += G.wpart[(size_t)q * G.GM * G.GN + e];
      a.grad[G.offW + i] = s;
    } else {
      const int n = i - G.K * G.N;
      const int Np = G.transposed ? G.GM : G.GN;
      for (int q = 0; q < G.bsplits; ++q) s += G.bpart[(size_t)q * Np + n];
      a.grad[G.offB + n] = s;
    }
  }
  if (l == 0 && blockIdx.x == 0 && threadIdx.x == 0 && a.loss_out) {
    float s = 0.0f;
    for (int i = 0; i < a.nloss; ++i) s += a.loss_partial[i];
    *a.loss_out = s;
  }
}

// Adam with bias correction: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// w -= lr (m / c1) / (sqrt(v / c2) + eps).
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int n, float lr,
                            float b1, float b2, float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
  const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__constant__ LayerDim kLayers[4] = {{IN, HID, K0P, HID, OFF_W0, OFF_B0},
                                    {HID, HID, HID, HID, OFF_W1, OFF_B1},
                                    {HID, HID, HID, HID, OFF_W2, OFF_B2},
                                    {HID, OUT, HID, N3P, OFF_W3, OFF_B3}};

// Tiled (TL) BF16 copies of the weights, zero padded: Wt[l] with element
// (n, k) = W_l[k][n] (rows = outputs: 256, or 16 for the output layer; K =
// inputs: 64 for layer 0, else 256), the B operand of the forward products;
// Wn[l] with element (k, n) = W_l[k][n] (rows = the 256 inputs; K = outputs,
// 64 for the output layer), the B operand of the input gradients (l >= 1).
__global__ void pack_kernel(const float* __restrict__ blob, PackedNet P) {
  const int l = blockIdx.y;
  const LayerDim& D = kLayers[l];
  const int rt = (l == 3) ? YN : HID, kt = (l == 0) ? XK : HID, kn = (l == 3) ? DYK : HID;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rt * kt; i += gridDim.x * blockDim.x) {
    const int n = i / kt, k = i % kt;
    const float w = (k < D.K && n < D.N) ? blob[D.offW + (size_t)k * D.N + n] : 0.0f;
    put_bf16(P.Wt[l], tl_off(n, k, rt), w);
  }
  if (l == 0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < HID * kn; i += gridDim.x * blockDim.x) {
    const int k = i / kn, n = i % kn;
    const float w = (n < D.N) ? blob[D.offW + (size_t)k * D.N + n] : 0.0f;
    put_bf16(P.Wn[l], tl_off(k, n, HID), w);
  }
}

// Weight initialisation: uniform(-sqrt(6/fan_in), +sqrt(6/fan_in)) from a
// SplitMix64 hash of (seed, index); biases zero.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__global__ void init_weights_kernel(float* __restrict__ blob, uint64_t seed) {
  const int l = blockIdx.y;
  const LayerDim& D = kLayers[l];
  const float bound = sqrtf(6.0f / (float)D.K);
  const int total = D.K * D.N + D.N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    if (i < D.K * D.N) {
      const uint64_t h = splitmix64(seed * 0x100000001B3ull + D.offW + i);
      const float u = (float)(h >> 40) * (1.0f / 16777216.0f);
      blob[D.offW + i] = bound * (2.0f * u - 1.0f);
    } else {
      blob[D.offB + (i - D.K * D.N)] = 0.0f;
    }
  }
}

// Normalisation statistics of the training set: mean and standard deviation
// of the 24 features (obs / Ic) and of the 10 targets, in FP64, deterministic
// (fixed per-thread strides, block tree, then one ordered sum).
constexpr int kStat = IN + OUT - 1;
__global__ void stats_partial_kernel(const float* __restrict__ obs,
                                     const float* __restrict__ params, int64_t n,
                                     double* __restrict__ part) {
  __shared__ double sh[256];
  double s[kStat], q[kStat];
  for (int j = 0; j < kStat; ++j) s[j] = q[j] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float* o = obs + i * IN;
    const float ic = ic_of(o);
    for (int j = 0; j < IN; ++j) {
      const double f = (double)(o[j] / ic);
      s[j] += f;
      q[j] += f * f;
    }
    float t[OUT - 1];
    targets(params + i * 10, ic, t);
    for (int j = 0; j < OUT - 1; ++j) {
      s[IN + j] += t[j];
      q[IN + j] += (double)t[j] * t[j];
    }
  }
  for (int j = 0; j < 2 * kStat; ++j) {
    sh[threadIdx.x] = (j < kStat) ? s[j] : q[j - kStat];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * 2 * kStat + j] = sh[0];
    __syncthreads();
  }
}
__global__ void stats_final_kernel(const double* __restrict__ part, int nblocks, int64_t n,
                                   float* __restrict__ blob) {
  const int j = threadIdx.x;
  if (j >= kStat) return;
  double s = 0.0, q = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    s += part[(size_t)b * 2 * kStat + j];
    q += part[(size_t)b * 2 * kStat + kStat + j];
  }
  const double mean = s / (double)n;
  const double var = fmax(q / (double)n - mean * mean, 0.0);
  const float sd = (float)fmax(sqrt(var), 1e-6);
  if (j < IN) {
    blob[OFF_INM + j] = (float)mean;
    blob[OFF_INS + j] = sd;
  } else {
    blob[OFF_OUTM + j - IN] = (float)mean;
    blob[OFF_OUTS + j - IN] = sd;
  }
}

// ---------------------------------------------------------------------------
// host side

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct Bufs {
  uint8_t *X0, *X0T, *H[3], *HT[3], *dY, *dYT, *dZ[3], *dZT[3];
  float *Z[3], *Y, *ic, *wpart[4], *bpart[4], *grad, *m, *v, *lossp;
  PackedNet P;
};

constexpr int kMaxLossBlocks = 4096;  // loss partials (256 rows each)

static Bufs carve(void* ws, int64_t M, size_t* used = nullptr) {
  char* p = (char*)ws;
  auto take = [&](size_t bytes) {
    void* r = p;
    p += (bytes + 255) & ~(size_t)255;
    return r;
  };
  Bufs b;
  take(infer_workspace_bytes());  // error word and packed inference weights
  b.X0 = (uint8_t*)take((size_t)M * XK * 2);
  b.X0T = (uint8_t*)take((size_t)M * XT * 2);
  for (int i = 0; i < 3; ++i) {
    b.Z[i] = (float*)take((size_t)M * HID * 4);
    b.H[i] = (uint8_t*)take((size_t)M * HID * 2);
    b.HT[i] = (uint8_t*)take((size_t)M * HID * 2);
    b.dZ[i] = (uint8_t*)take((size_t)M * HID * 2);
    b.dZT[i] = (uint8_t*)take((size_t)M * HID * 2);
  }
  b.Y = (float*)take((size_t)M * YN * 4);
  b.dY = (uint8_t*)take((size_t)M * DYK * 2);
  b.dYT = (uint8_t*)take((size_t)M * YN * 2);
  b.ic = (float*)take((size_t)M * 4);
  for (int l = 0; l < 4; ++l) {
    b.wpart[l] = (float*)take((size_t)kSplits * HID * HID * 4);
    b.bpart[l] = (float*)take((size_t)kSplits * HID * 4);
  }
  b.grad = (float*)take(NBLOB * 4);
  b.m = (float*)take(NBLOB * 4);
  b.v = (float*)take(NBLOB * 4);
  b.lossp = (float*)take(kMaxLossBlocks * 4);
  for (int l = 0; l < 4; ++l) {
    b.P.Wt[l] = (uint8_t*)take((size_t)(l == 3 ? YN : HID) * (l == 0 ? XK : HID) * 2);
    b.P.Wn[l] = (uint8_t*)take((size_t)HID * (l == 3 ? DYK : HID) * 2);
  }
  if (used) *used = (size_t)(p - (char*)ws);
  return b;
}

size_t workspace_bytes(int64_t rows) {
  size_t used = 0;
  carve(nullptr, padded_rows(rows), &used);
  const size_t stats = infer_workspace_bytes() + (size_t)256 * 2 * (IN + OUT - 1) * sizeof(double);
  return used > stats ? used : stats;
}

// batch rows padded to the 128-row tiles of the products
int64_t padded_rows(int64_t n) { return round_up(n > 0 ? n : 1, 128); }

static cudaError_t pack(const float* blob, const PackedNet& P, cudaStream_t s) {
  pack_kernel<<<dim3(64, 4), 256, 0, s>>>(blob, P);
  return cudaGetLastError();
}

static TcGemmArgs gemm_args(const uint8_t* A, int64_t MA, const uint8_t* B, int64_t NB, int K,
                            int* err) {
  TcGemmArgs g{};
  g.A = A;
  g.MA = MA;
  g.B = B;
  g.NB = NB;
  g.K = K;
  g.kchunks_per_split = K / 64;
  g.err = err;
  return g;
}

// Forward pass over M (padded) rows whose features are already in X0.
static cudaError_t forward(const float* blob, const Bufs& b, int64_t M, int* err, cudaStream_t s) {
  cudaError_t e;
  const uint8_t* in = b.X0;
  int kin = XK;
  const int mt = (int)(M / 128);
  for (int l = 0; l < 3; ++l) {
    TcGemmArgs g = gemm_args(in, M, b.P.Wt[l], HID, kin, err);
    g.bias = blob + kLayersHost[l].offB;
    g.Z = b.Z[l];
    g.ldz = HID;
    g.H = b.H[l];
    g.HT = b.HT[l];
    if ((e = tc_gemm(g, HID, EPI_HIDDEN, mt, 1, s)) != cudaSuccess) return e;
    in = b.H[l];
    kin = HID;
  }
  TcGemmArgs g = gemm_args(b.H[2], M, b.P.Wt[3], YN, HID, err);
  g.bias = blob + OFF_B3;
  g.n_valid = OUT;
  g.Z = b.Y;
  g.ldz = YN;
  return tc_gemm(g, YN, EPI_OUT, mt, 1, s);
}

// Split of a batch-long K (M rows, 64 per chunk) over at most kSplits CTAs
// per tile, every split owning at least one chunk.
static void batch_split(int64_t M, int* per, int* splits) {
  const int64_t total = M / 64;
  const int64_t want = total < kSplits ? total : kSplits;
  *per = (int)((total + want - 1) / want);
  *splits = (int)((total + *per - 1) / *per);
}

// Backward pass for a batch of M rows (dY already written): weight and bias
// gradients into b.grad, in blob layout.
static cudaError_t backward(const Bufs& b, int64_t M, float* loss_out, int nloss, int* err,
                            cudaStream_t s) {
  cudaError_t e;
  const int mt = (int)(M / 128);
  int per = 1, S = 1;
  batch_split(M, &per, &S);
  // bias-gradient batch columns per split (whole 64-column blocks)
  const int64_t bchunk = ((M + kSplits - 1) / kSplits + 63) / 64 * 64;
  const int SB = (int)((M + bchunk - 1) / bchunk);
  // input gradient of layer l (l = 3, 2, 1): dZ_{l-1} = (dZ_l W_l^T) * GELU'(Z_{l-1})
  auto dx = [&](int l, const uint8_t* dOut, int kout, uint8_t* H, uint8_t* HT) {
    TcGemmArgs g = gemm_args(dOut, M, b.P.Wn[l], HID, kout, err);
    g.Zprev = b.Z[l - 1];
    g.ldzp = HID;
    g.H = H;
    g.HT = HT;
    return tc_gemm(g, HID, EPI_DX, mt, 1, s);
  };
  // weight gradient: D[256][n] = A^T-rows x B^T-rows over the batch, split-K
  auto dw = [&](int l, const uint8_t* AT, const uint8_t* BT, int n) {
    TcGemmArgs g = gemm_args(AT, HID, BT, n, (int)M, err);
    g.kchunks_per_split = per;
    g.P = b.wpart[l];
    return tc_gemm(g, n, EPI_PARTIAL, HID / 128, S, s);
  };
  auto bias = [&](int l, const uint8_t* GT, int n) {
    rowsum_kernel<<<dim3(n / 8, SB), 32, 0, s>>>(GT, n, M, bchunk, b.bpart[l]);
    return cudaGetLastError();
  };
  if ((e = dx(3, b.dY, DYK, b.dZ[2], b.dZT[2])) != cudaSuccess) return e;
  if ((e = dw(3, b.HT[2], b.dYT, YN)) != cudaSuccess) return e;
  if ((e = bias(3, b.dYT, YN)) != cudaSuccess) return e;
  if ((e = dx(2, b.dZ[2], HID, b.dZ[1], b.dZT[1])) != cudaSuccess) return e;
  if ((e = dw(2, b.HT[1], b.dZT[2], HID)) != cudaSuccess) return e;
  if ((e = bias(2, b.dZT[2], HID)) != cudaSuccess) return e;
  if ((e = dx(1, b.dZ[1], HID, nullptr, b.dZT[0])) != cudaSuccess) return e;
  if ((e = dw(1, b.HT[0], b.dZT[1], HID)) != cudaSuccess) return e;
  if ((e = bias(1, b.dZT[1], HID)) != cudaSuccess) return e;
  // layer 0 transposed: dW0^T[n][k] = sum_m dZ0[m][n] X0[m][k]
  if ((e = dw(0, b.dZT[0], b.X0T, XT)) != cudaSuccess) return e;
  if ((e = bias(0, b.dZT[0], HID)) != cudaSuccess) return e;
  GradArgs ga{};
  ga.L[0] = GradLayer{b.wpart[0], b.bpart[0], HID, XT, IN, HID, 1, S, SB, OFF_W0, OFF_B0};
  ga.L[1] = GradLayer{b.wpart[1], b.bpart[1], HID, HID, HID, HID, 0, S, SB, OFF_W1, OFF_B1};
  ga.L[2] = GradLayer{b.wpart[2], b.bpart[2], HID, HID, HID, HID, 0, S, SB, OFF_W2, OFF_B2};
  ga.L[3] = GradLayer{b.wpart[3], b.bpart[3], HID, YN, HID, OUT, 0, S, SB, OFF_W3, OFF_B3};
  ga.grad = b.grad;
  ga.loss_partial = b.lossp;
  ga.nloss = nloss;
  ga.loss_out = loss_out;
  reduce_grad_kernel<<<dim3(128, 4), 256, 0, s>>>(ga);
  return cudaGetLastError();
}

static cudaError_t loss_and_dy(const Bufs& b, int64_t rows, int64_t M, Perm perm,
                               const float* params, const float* blob, int* nloss,
                               cudaStream_t s) {
  const int nb = (int)((M + 255) / 256);
  if (nb > kMaxLossBlocks) return cudaErrorInvalidValue;
  loss_kernel<<<nb, 256, 0, s>>>(b.Y, rows, M, perm, params, b.ic, blob, b.dY, b.dYT, b.lossp);
  *nloss = nb;
  return cudaGetLastError();
}

cudaError_t nn_init(void* ws, float* blob, const float* obs, const float* params, int64_t n,
                    uint64_t seed, cudaStream_t s) {
  init_weights_kernel<<<dim3(64, 4), 256, 0, s>>>(blob, seed);
  const int nb = 256;
  double* part = (double*)((char*)ws + infer_workspace_bytes());  // after the error word
  stats_partial_kernel<<<nb, 256, 0, s>>>(obs, params, n, part);
  stats_final_kernel<<<1, 64, 0, s>>>(part, nb, n, blob);
  return cudaGetLastError();
}

cudaError_t nn_grad(void* ws, const float* blob, const float* obs, const float* params,
                    int64_t n, float* grad_out, float* loss_out, cudaStream_t s) {
  const int64_t M = padded_rows(n);
  Bufs b = carve(ws, M);
  cudaError_t e;
  if ((e = pack(blob, b.P, s)) != cudaSuccess) return e;
  Perm id{1, 0, 0, n};
  int* err = static_cast<int*>(ws);
  features_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(obs, n, M, id, blob, b.X0, b.X0T,
                                                              b.ic);
  if ((e = forward(blob, b, M, err, s)) != cudaSuccess) return e;
  int nloss = 0;
  if ((e = loss_and_dy(b, n, M, id, params, blob, &nloss, s)) != cudaSuccess) return e;
  if ((e = backward(b, M, loss_out, nloss, err, s)) != cudaSuccess) return e;
  return cudaMemcpyAsync(grad_out, b.grad, NTRAIN * sizeof(float), cudaMemcpyDeviceToDevice, s);
}

cudaError_t nn_train(void* ws, float* blob, const float* obs, const float* params, int64_t n,
                     int batch, int epochs, float lr0, uint64_t seed, float* loss_hist,
                     cudaStream_t s) {
  const int64_t M = batch;
  Bufs b = carve(ws, M);
  int* err = static_cast<int*>(ws);
  cudaError_t e;
  if ((e = cudaMemsetAsync(b.m, 0, NBLOB * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b.v, 0, NBLOB * 4, s)) != cudaSuccess) return e;
  const int64_t spe = n / batch;
  const int64_t total = spe * epochs;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  double p1 = 1.0, p2 = 1.0;
  for (int64_t t = 0; t < total; ++t) {
    const int64_t ep = t / spe, bi = t % spe;
    // a different affine permutation of the training set every epoch
    uint64_t h = seed * 0x9E3779B97F4A7C15ull + (uint64_t)ep * 0xD1B54A32D192ED03ull + 1;
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
    auto gcd = [](uint64_t a, uint64_t c) {
      while (c) {
        const uint64_t r = a % c;
        a = c;
        c = r;
      }
      return a;
    };
    uint64_t mult = (n > 1) ? 1 + h % (uint64_t)(n - 1) : 1;
    while (n > 1 && gcd(mult, (uint64_t)n) != 1) mult = mult % (uint64_t)(n - 1) + 1;
    Perm perm{mult, (h >> 17) % (uint64_t)n, bi * batch, n};
    if ((e = pack(blob, b.P, s)) != cudaSuccess) return e;
    features_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(obs, M, M, perm, blob, b.X0,
                                                                b.X0T, b.ic);
    if ((e = forward(blob, b, M, err, s)) != cudaSuccess) return e;
    int nloss = 0;
    if ((e = loss_and_dy(b, M, M, perm, params, blob, &nloss, s)) != cudaSuccess) return e;
    if ((e = backward(b, M, loss_hist ? loss_hist + t : nullptr, nloss, err, s)) != cudaSuccess)
      return e;
    const double lr = lr0 * 0.5 * (1.0 + cos(3.14159265358979323846 * (double)t / (double)total));
    p1 *= b1;
    p2 *= b2;
    adam_kernel<<<(int)((NTRAIN + 255) / 256), 256, 0, s>>>(
        blob, b.grad, b.m, b.v, (int)NTRAIN, (float)lr, b1, b2, (float)(1.0 - p1),
        (float)(1.0 - p2), eps);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace nn
}  // namespace vfisv
