// Initial-guess network (Sec. 5): a 24-256-256-256-11 multilayer perceptron
// with GELU activations, trained and evaluated by hand-written BF16
// tensor-core kernels (mma.sync m16n8k16, FP32 accumulation, operands staged
// in shared memory by cp.async and fed with ldmatrix).
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

namespace vfisv {
namespace nn {

using bf16 = __nv_bfloat16;

__constant__ LayerDim kLayers[4] = {{IN, HID, K0P, HID, OFF_W0, OFF_B0},
                                    {HID, HID, HID, HID, OFF_W1, OFF_B1},
                                    {HID, HID, HID, HID, OFF_W2, OFF_B2},
                                    {HID, OUT, HID, N3P, OFF_W3, OFF_B3}};

// ---------------------------------------------------------------------------
// small PTX helpers

__device__ __forceinline__ void cp_async16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// Tiled GEMM C[M,N] = sum_k A(m,k) B(k,n), BF16 in, FP32 accumulate.
// A is stored [M][K] (AK = true) or [K][M]; B is stored [N][K] (BKM = true) or
// [K][N].  M % 128 == 0, N % 64 == 0, K % 32 == 0 (callers pad).  blockIdx.z
// selects a K chunk of length kchunk (split-K for the weight gradients).

constexpr int BM = 128, BN = 64, BK = 32, GT = 128;
enum Epi { EPI_HIDDEN = 0, EPI_OUT = 1, EPI_DX_GELU = 2, EPI_PARTIAL = 3 };

struct GemmArgs {
  const bf16* A;
  int lda;
  const bf16* B;
  int ldb;
  int M, N, K, kchunk;
  const float* bias;
  int n_valid;
  float* Z;  // HIDDEN: pre-activation; OUT: output; PARTIAL: [split][M][N]
  int ldz;
  bf16* H;   // HIDDEN: GELU(Z); DX_GELU: dZ of the layer input
  int ldh;
  const float* Zprev;  // DX_GELU: pre-activation of the layer input
  int ldzp;
};

template <bool AK, bool BKM, int EPI>
__global__ void __launch_bounds__(GT) gemm_kernel(GemmArgs g) {
  constexpr int SA = AK ? BM * (BK + 8) : BK * (BM + 8);
  constexpr int SB = BKM ? BN * (BK + 8) : BK * (BN + 8);
  __shared__ __align__(16) bf16 sA[2][SA];
  __shared__ __align__(16) bf16 sB[2][SB];
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = (warp >> 1) * 64, wn = (warp & 1) * 32;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;

  auto load_tile = [&](int st, int k0) {
    if (AK) {
      for (int c = tid; c < BM * BK / 8; c += GT) {
        const int r = c / (BK / 8), cc = (c % (BK / 8)) * 8;
        cp_async16(&sA[st][r * (BK + 8) + cc], g.A + (size_t)(m0 + r) * g.lda + k0 + cc);
      }
    } else {
      for (int c = tid; c < BK * BM / 8; c += GT) {
        const int r = c / (BM / 8), cc = (c % (BM / 8)) * 8;
        cp_async16(&sA[st][r * (BM + 8) + cc], g.A + (size_t)(k0 + r) * g.lda + m0 + cc);
      }
    }
    if (BKM) {
      for (int c = tid; c < BN * BK / 8; c += GT) {
        const int r = c / (BK / 8), cc = (c % (BK / 8)) * 8;
        cp_async16(&sB[st][r * (BK + 8) + cc], g.B + (size_t)(n0 + r) * g.ldb + k0 + cc);
      }
    } else {
      for (int c = tid; c < BK * BN / 8; c += GT) {
        const int r = c / (BN / 8), cc = (c % (BN / 8)) * 8;
        cp_async16(&sB[st][r * (BN + 8) + cc], g.B + (size_t)(k0 + r) * g.ldb + n0 + cc);
      }
    }
    cp_async_commit();
  };

  const int nk = (kend - kbeg) / BK;
  if (nk > 0) load_tile(0, kbeg);
  for (int t = 0; t < nk; ++t) {
    if (t + 1 < nk) {
      load_tile((t + 1) & 1, kbeg + (t + 1) * BK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const bf16* a = sA[t & 1];
    const bf16* b = sB[t & 1];
#pragma unroll
    for (int kk = 0; kk < BK / 16; ++kk) {
      uint32_t af[4][4], bfr[4][2];
      const int j = lane >> 3, r = lane & 7;
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) {
        const int mb = j & 1, kb = j >> 1;
        if (AK)
          ldsm_x4(af[mi], a + (wm + mi * 16 + mb * 8 + r) * (BK + 8) + kk * 16 + kb * 8);
        else
          ldsm_x4_t(af[mi], a + (kk * 16 + kb * 8 + r) * (BM + 8) + wm + mi * 16 + mb * 8);
      }
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        const int nb = j >> 1, kb = j & 1;
        uint32_t q[4];
        if (BKM)
          ldsm_x4(q, b + (wn + (2 * np + nb) * 8 + r) * (BK + 8) + kk * 16 + kb * 8);
        else
          ldsm_x4_t(q, b + (kk * 16 + kb * 8 + r) * (BN + 8) + wn + (2 * np + nb) * 8);
        bfr[2 * np][0] = q[0];
        bfr[2 * np][1] = q[1];
        bfr[2 * np + 1][0] = q[2];
        bfr[2 * np + 1][1] = q[3];
      }
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni][0], bfr[ni][1]);
    }
    __syncthreads();
  }

  // epilogue: thread holds rows (lane/4, +8) and column pairs ((lane%4)*2)
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int row = m0 + wm + mi * 16 + (lane >> 2) + hh * 8;
        const int col = n0 + wn + ni * 8 + (lane & 3) * 2;
        float v0 = acc[mi][ni][2 * hh], v1 = acc[mi][ni][2 * hh + 1];
        if (EPI == EPI_HIDDEN) {
          v0 += g.bias[col];
          v1 += g.bias[col + 1];
          *reinterpret_cast<float2*>(g.Z + (size_t)row * g.ldz + col) = make_float2(v0, v1);
          *reinterpret_cast<__nv_bfloat162*>(g.H + (size_t)row * g.ldh + col) =
              __floats2bfloat162_rn(gelu(v0), gelu(v1));
        } else if (EPI == EPI_OUT) {
          v0 += (col < g.n_valid) ? g.bias[col] : 0.0f;
          v1 += (col + 1 < g.n_valid) ? g.bias[col + 1] : 0.0f;
          *reinterpret_cast<float2*>(g.Z + (size_t)row * g.ldz + col) = make_float2(v0, v1);
        } else if (EPI == EPI_DX_GELU) {
          const float2 zp = *reinterpret_cast<const float2*>(g.Zprev + (size_t)row * g.ldzp + col);
          *reinterpret_cast<__nv_bfloat162*>(g.H + (size_t)row * g.ldh + col) =
              __floats2bfloat162_rn(v0 * gelu_grad(zp.x), v1 * gelu_grad(zp.y));
        } else {
          float* P = g.Z + (size_t)blockIdx.z * g.M * g.N;
          *reinterpret_cast<float2*>(P + (size_t)row * g.N + col) = make_float2(v0, v1);
        }
      }
}

template <bool AK, bool BKM, int EPI>
static cudaError_t gemm(const GemmArgs& g, int splits, cudaStream_t s) {
  dim3 grid(g.M / BM, g.N / BN, splits);
  gemm_kernel<AK, BKM, EPI><<<grid, GT, 0, s>>>(g);
  return cudaGetLastError();
}

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

__global__ void features_kernel(const float* __restrict__ obs, int64_t rows, int64_t mpad,
                                Perm perm, const float* __restrict__ blob,
                                bf16* __restrict__ X, float* __restrict__ ic_out) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= mpad) return;
  bf16* x = X + m * K0P;
  if (m >= rows) {
    for (int j = 0; j < K0P; ++j) x[j] = __float2bfloat16(0.0f);
    ic_out[m] = 1.0f;
    return;
  }
  const int64_t s = sample_of(m, perm);
  const float* o = obs + s * IN;
  const float ic = ic_of(o);
  const float inv = 1.0f / ic;
  for (int j = 0; j < IN; ++j)
    x[j] = __float2bfloat16((o[j] * inv - blob[OFF_INM + j]) / blob[OFF_INS + j]);
  for (int j = IN; j < K0P; ++j) x[j] = __float2bfloat16(0.0f);
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

// Loss of Sec. 5's regression plus the confidence output, and dL/dy.
__global__ void loss_kernel(const float* __restrict__ Y, int64_t rows, int64_t mpad, Perm perm,
                            const float* __restrict__ params, const float* __restrict__ ic,
                            const float* __restrict__ blob, bf16* __restrict__ dY,
                            float* __restrict__ partial) {
  __shared__ float red[256];
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (m < mpad) {
    bf16* d = dY + m * N3P;
    if (m < rows) {
      const int64_t s = sample_of(m, perm);
      float t[OUT - 1];
      targets(params + s * 10, ic[m], t);
      const float* y = Y + m * N3P;
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
      for (int o = 0; o < OUT - 1; ++o) d[o] = __float2bfloat16(2.0f * e[o] * invn / (OUT - 1));
      d[OUT - 1] = __float2bfloat16(2.0f * ec * invn);
      for (int o = OUT; o < N3P; ++o) d[o] = __float2bfloat16(0.0f);
    } else {
      for (int o = 0; o < N3P; ++o) d[o] = __float2bfloat16(0.0f);
    }
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Column sums of dZ [M][N] (bias gradients) in row chunks: partial[s][N].
__global__ void colsum_kernel(const bf16* __restrict__ dZ, int M, int N, int chunk,
                              float* __restrict__ partial) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int s = blockIdx.y;
  float acc = 0.0f;
  for (int m = s * chunk; m < min(M, (s + 1) * chunk); ++m)
    acc += __bfloat162float(dZ[(size_t)m * N + n]);
  partial[(size_t)s * N + n] = acc;
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

// BF16 copies of the weights: Wt [Np][Kp] (forward) and Wn [Kp][Np] (input
// gradient), zero padded.
__global__ void pack_kernel(const float* __restrict__ blob, PackedNet P) {
  const int l = blockIdx.y;
  const LayerDim& D = kLayers[l];
  const int total = D.Kp * D.Np;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int k = i / D.Np, n = i % D.Np;
    const float w = (k < D.K && n < D.N) ? blob[D.offW + (size_t)k * D.N + n] : 0.0f;
    P.Wn[l][(size_t)k * D.Np + n] = __float2bfloat16(w);
    P.Wt[l][(size_t)n * D.Kp + k] = __float2bfloat16(w);
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
  bf16 *X0, *H[3], *dY, *dZ[2];
  float *Z[3], *Y, *ic, *wpart[4], *bpart[4], *grad, *m, *v, *lossp;
  PackedNet P;
};

static Bufs carve(void* ws, int64_t M, size_t* used = nullptr) {
  char* p = (char*)ws;
  auto take = [&](size_t bytes) {
    void* r = p;
    p += (bytes + 255) & ~(size_t)255;
    return r;
  };
  Bufs b;
  take(infer_workspace_bytes());  // error word and packed inference weights
  b.X0 = (bf16*)take((size_t)M * K0P * 2);
  for (int i = 0; i < 3; ++i) {
    b.Z[i] = (float*)take((size_t)M * HID * 4);
    b.H[i] = (bf16*)take((size_t)M * HID * 2);
  }
  b.Y = (float*)take((size_t)M * N3P * 4);
  b.dY = (bf16*)take((size_t)M * N3P * 2);
  b.dZ[0] = (bf16*)take((size_t)M * HID * 2);
  b.dZ[1] = (bf16*)take((size_t)M * HID * 2);
  b.ic = (float*)take((size_t)M * 4);
  for (int l = 0; l < 4; ++l) {
    b.wpart[l] = (float*)take((size_t)kSplits * HID * HID * 4);
    b.bpart[l] = (float*)take((size_t)kSplits * HID * 4);
  }
  b.grad = (float*)take(NBLOB * 4);
  b.m = (float*)take(NBLOB * 4);
  b.v = (float*)take(NBLOB * 4);
  b.lossp = (float*)take(4096 * 4);
  for (int l = 0; l < 4; ++l) {
    b.P.Wt[l] = (bf16*)take((size_t)kLayersHost[l].Kp * kLayersHost[l].Np * 2);
    b.P.Wn[l] = (bf16*)take((size_t)kLayersHost[l].Kp * kLayersHost[l].Np * 2);
  }
  if (used) *used = (size_t)(p - (char*)ws);
  return b;
}

size_t workspace_bytes(int64_t rows) {
  size_t used = 0;
  carve(nullptr, round_up(rows, BM), &used);
  const size_t stats = infer_workspace_bytes() + (size_t)256 * 2 * (IN + OUT - 1) * sizeof(double);
  return used > stats ? used : stats;
}

int64_t padded_rows(int64_t n) { return round_up(n > 0 ? n : 1, (int64_t)kSplits * BK); }

static cudaError_t pack(const float* blob, const PackedNet& P, cudaStream_t s) {
  pack_kernel<<<dim3(64, 4), 256, 0, s>>>(blob, P);
  return cudaGetLastError();
}

// Forward pass over M (padded) rows whose features are already in X0.
static cudaError_t forward(const float* blob, const Bufs& b, int64_t M, cudaStream_t s) {
  cudaError_t e;
  const bf16* in = b.X0;
  int kin = K0P;
  for (int l = 0; l < 3; ++l) {
    GemmArgs g{};
    g.A = in; g.lda = kin;
    g.B = b.P.Wt[l]; g.ldb = kin;
    g.M = (int)M; g.N = HID; g.K = kin; g.kchunk = kin;
    g.bias = blob + kLayersHost[l].offB;
    g.Z = b.Z[l]; g.ldz = HID;
    g.H = b.H[l]; g.ldh = HID;
    if ((e = gemm<true, true, EPI_HIDDEN>(g, 1, s)) != cudaSuccess) return e;
    in = b.H[l];
    kin = HID;
  }
  GemmArgs g{};
  g.A = b.H[2]; g.lda = HID;
  g.B = b.P.Wt[3]; g.ldb = HID;
  g.M = (int)M; g.N = N3P; g.K = HID; g.kchunk = HID;
  g.bias = blob + OFF_B3;
  g.n_valid = OUT;
  g.Z = b.Y; g.ldz = N3P;
  return gemm<true, true, EPI_OUT>(g, 1, s);
}

// Backward pass for a batch of M rows (dY already written): weight and bias
// gradients into b.grad, in blob layout.
static cudaError_t backward(const Bufs& b, int64_t M, float* loss_out, int nloss,
                            cudaStream_t s) {
  cudaError_t e;
  const int chunk = (int)(M / kSplits);  // M % (kSplits * BK) == 0 by construction
  const bf16* dOut = b.dY;
  int nOut = N3P;
  GradArgs ga{};
  for (int l = 3; l >= 0; --l) {
    const LayerDim& D = kLayersHost[l];
    const bf16* Hin = (l == 0) ? b.X0 : b.H[l - 1];
    const int kin = D.Kp;
    // weight gradient: dW = H_in^T dOut (layer 0 computed transposed: dOut^T X0)
    GemmArgs g{};
    if (l == 0) {
      g.A = dOut; g.lda = nOut;  // A(i = n, c = m) stored [m][n]
      g.B = Hin; g.ldb = kin;    // B(c = m, j = k) stored [m][k]
      g.M = nOut; g.N = kin;
    } else {
      g.A = Hin; g.lda = kin;
      g.B = dOut; g.ldb = nOut;
      g.M = kin; g.N = nOut;
    }
    g.K = (int)M; g.kchunk = chunk;
    g.Z = b.wpart[l];
    if ((e = gemm<false, false, EPI_PARTIAL>(g, kSplits, s)) != cudaSuccess) return e;
    colsum_kernel<<<dim3((nOut + 127) / 128, kSplits), 128, 0, s>>>(dOut, (int)M, nOut, chunk,
                                                                    b.bpart[l]);
    ga.L[l] = GradLayer{b.wpart[l], b.bpart[l], g.M, g.N, D.K, D.N, l == 0 ? 1 : 0,
                        kSplits, kSplits, D.offW, D.offB};
    if (l > 0) {
      // input gradient through the GELU of the layer below
      GemmArgs d{};
      d.A = dOut; d.lda = nOut;
      d.B = b.P.Wn[l]; d.ldb = nOut;
      d.M = (int)M; d.N = kin; d.K = nOut; d.kchunk = nOut;
      d.Zprev = b.Z[l - 1]; d.ldzp = HID;
      bf16* dst = b.dZ[l & 1];
      d.H = dst; d.ldh = HID;
      if ((e = gemm<true, true, EPI_DX_GELU>(d, 1, s)) != cudaSuccess) return e;
      dOut = dst;
      nOut = HID;
    }
  }
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
  loss_kernel<<<nb, 256, 0, s>>>(b.Y, rows, M, perm, params, b.ic, blob, b.dY, b.lossp);
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
  features_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(obs, n, M, id, blob, b.X0, b.ic);
  if ((e = forward(blob, b, M, s)) != cudaSuccess) return e;
  int nloss = 0;
  if ((e = loss_and_dy(b, n, M, id, params, blob, &nloss, s)) != cudaSuccess) return e;
  if ((e = backward(b, M, loss_out, nloss, s)) != cudaSuccess) return e;
  return cudaMemcpyAsync(grad_out, b.grad, NTRAIN * sizeof(float), cudaMemcpyDeviceToDevice, s);
}

cudaError_t nn_train(void* ws, float* blob, const float* obs, const float* params, int64_t n,
                     int batch, int epochs, float lr0, uint64_t seed, float* loss_hist,
                     cudaStream_t s) {
  const int64_t M = batch;
  Bufs b = carve(ws, M);
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
                                                                b.ic);
    if ((e = forward(blob, b, M, s)) != cudaSuccess) return e;
    int nloss = 0;
    if ((e = loss_and_dy(b, M, M, perm, params, blob, &nloss, s)) != cudaSuccess) return e;
    if ((e = backward(b, M, loss_hist ? loss_hist + t : nullptr, nloss, s)) != cudaSuccess)
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
