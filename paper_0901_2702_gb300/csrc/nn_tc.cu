// Training GEMMs of the initial-guess network (Sec. 5) on the fifth-generation
// tensor cores.  Every product of the forward and backward passes is one
// launch of tc_gemm_kernel: a CTA computes a 128-row tile of D = A B^T over a
// range of K (split-K for the weight gradients), BF16 operands streamed by 1D
// bulk copies through a four-stage shared-memory ring, FP32 accumulators in
// tensor memory, and an epilogue (16 warps, each a quarter of the
// accumulator lanes -- one row per thread -- and a quarter of the columns)
// that writes the next product's operands directly.
//
// Operand layout in global memory, "tiled canonical" TL(R, C) for an R x C
// BF16 matrix (R a multiple of 8, C of 64): K-chunks of 64 columns one after
// the other, inside a chunk 8-row groups of 1024 bytes, inside a group eight
// 128-byte core matrices along K, each 8 rows x 16 bytes.  A chunk of an
// operand tile is then one contiguous block whose shared-memory copy is the
// no-swizzle K-major layout of the MMA descriptors (leading-dimension byte
// offset 128, stride-dimension byte offset 1024).  Products that contract
// over the batch (weight gradients) take the transposed activations and
// gradients, which the producing epilogues write beside the plain ones.
//
// Every wait is bounded (about 1 s); on a timeout the kernel lets the copies
// and tensor-core work it issued finish (bounded again), frees its tensor
// memory, writes kDevErrNnWait to the error word and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"
#include "nn.cuh"
#include "nn_device.cuh"
#include "nn_tc.cuh"
#include "tc_device.cuh"

namespace vfisv {
namespace nn {

namespace {

using bf16 = __nv_bfloat16;

constexpr int TMR = 128;      // rows of a D tile (MMA M)
constexpr int KCH = 64;       // K per stage
constexpr int NSTAGE = 4;     // ring depth
constexpr uint32_t kAChunk = TMR * KCH * 2;  // 16384

constexpr int kThreads = 512;  // 16 warps: 4 accumulator lane quarters x 4 column quarters

template <int N, int EPI>
__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(TcGemmArgs g) {
  static_assert(N == 16 || N == 32 || N == 256, "tile width");
  constexpr uint32_t kBChunk = N * KCH * 2;
  constexpr uint32_t kStage = kAChunk + kBChunk;
  constexpr int kTmemCols = N < 32 ? 32 : N;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sb = smem_u32(sm);
  const uint32_t bar_full = sb + NSTAGE * kStage, bar_empty = bar_full + 8 * NSTAGE,
                 bar_mma = bar_empty + 8 * NSTAGE;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + NSTAGE * kStage + 16 * NSTAGE + 8);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int mt = blockIdx.x, split = blockIdx.y;
  const int kc0 = split * g.kchunks_per_split;
  int nk = g.K / KCH - kc0;
  if (nk > g.kchunks_per_split) nk = g.kchunks_per_split;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 2 * NSTAGE + 1; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_full + 8 * i), "r"(1)
                   : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = *tmem_slot;

  // issuer: loads of stage i go to slot i % NSTAGE; the slot is refilled once
  // the MMAs that read it have completed (their commit on the empty barrier)
  bool bad = false;
  int loaded = 0, consumed = 0;
  if (tid == 0) {
    auto load = [&](int i) {
      const int slot = i % NSTAGE, kc = kc0 + i;
      const uint32_t dst = sb + slot * kStage, bar = bar_full + 8 * slot;
      expect_tx(bar, kStage);
      bulk_load(dst, g.A + (size_t)kc * g.MA * (KCH * 2) + (size_t)mt * kAChunk, kAChunk, bar);
      bulk_load(dst + kAChunk, g.B + (size_t)kc * g.NB * (KCH * 2), kBChunk, bar);
    };
    for (; loaded < NSTAGE && loaded < nk; ++loaded) load(loaded);
    constexpr uint32_t idesc = idesc_bf16(TMR, N);
    for (int i = 0; i < nk && !bad; ++i) {
      const int slot = i % NSTAGE;
      if (!mbar_wait(bar_full + 8 * slot, (i / NSTAGE) & 1)) {
        bad = true;
        break;
      }
      consumed = i + 1;
      tc_after_sync();
      const uint32_t sa = sb + slot * kStage, sbb = sa + kAChunk;
#pragma unroll
      for (int ks = 0; ks < KCH / 16; ++ks)
        mma_bf16(tmem, sdesc(sa + ks * 256, 128, 1024), sdesc(sbb + ks * 256, 128, 1024), idesc,
                 (i | ks) != 0);
      mma_commit(bar_empty + 8 * slot);
      if (i + NSTAGE < nk) {
        if (!mbar_wait(bar_empty + 8 * slot, (i / NSTAGE) & 1)) {
          bad = true;
          break;
        }
        load(loaded++);
      }
    }
    mma_commit(bar_mma);  // tracks every MMA issued above
  }
  const bool ok_mma = mbar_wait(bar_mma, 0);
  if (tid == 0 && ok_mma && !bad) {
    // the tensor cores' last arrivals on the slot barriers precede the exit
    for (int i = consumed > NSTAGE ? consumed - NSTAGE : 0; i < consumed; ++i)
      mbar_wait(bar_empty + 8 * (i % NSTAGE), (i / NSTAGE) & 1);
  }
  if (__syncthreads_or(!ok_mma || (tid == 0 && bad))) {
    if (tid == 0) {
      // let the copies issued but not consumed land before the memory is released
      for (int i = consumed; i < loaded; ++i) mbar_wait(bar_full + 8 * (i % NSTAGE), (i / NSTAGE) & 1);
      atomicExch(g.err, kDevErrNnWait);
    }
  } else {
    tc_after_sync();
    // warp w reads accumulator lanes 32 (w % 4) .. + 31 (its lane quarter)
    // and the column quarter w / 4 (for N <= 32 the first quarter takes all)
    const int lq = warp & 3, cq = warp >> 2;
    const int row = 32 * lq + (tid & 31);  // accumulator lane = tile row
    const int64_t m = (int64_t)mt * TMR + row;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * lq) << 16);
    constexpr int kCols = N >= 128 ? N / 4 : N;  // columns per warp
    const int cbeg = (N >= 128) ? cq * kCols : 0;
    const bool active = (N >= 128) || cq == 0;
    if constexpr (N == 16) {
      if (!active) goto done;
      float v[16];
      tmem_ld16(lane_addr, v);
      if constexpr (EPI == EPI_OUT) {
        float* z = g.Z + m * g.ldz;
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(z + j) =
              make_float4(v[j] + (j < g.n_valid ? g.bias[j] : 0.0f),
                          v[j + 1] + (j + 1 < g.n_valid ? g.bias[j + 1] : 0.0f),
                          v[j + 2] + (j + 2 < g.n_valid ? g.bias[j + 2] : 0.0f),
                          v[j + 3] + (j + 3 < g.n_valid ? g.bias[j + 3] : 0.0f));
      } else {  // EPI_PARTIAL
        float* pp = g.P + ((size_t)split * g.MA + m) * N;
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(pp + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      }
    } else {
      if (!active) goto done;
#pragma unroll 1
      for (int c0 = cbeg; c0 < cbeg + kCols; c0 += 32) {
        float v[32];
        tmem_ld32(lane_addr + (uint32_t)c0, v);
        if constexpr (EPI == EPI_PARTIAL) {
          float* pp = g.P + ((size_t)split * g.MA + m) * N + c0;
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            *reinterpret_cast<float4*>(pp + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        } else {
          // EPI_HIDDEN: z = acc + bias, h = GELU(z); EPI_DX: d = acc GELU'(z_prev)
          float h[32];
          if constexpr (EPI == EPI_HIDDEN) {
            float* z = g.Z + m * g.ldz + c0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float zz = v[j] + g.bias[c0 + j];
              v[j] = zz;
              h[j] = gelu(zz);
            }
#pragma unroll
            for (int j = 0; j < 32; j += 4)
              *reinterpret_cast<float4*>(z + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
          } else {
            const float* zp = g.Zprev + m * g.ldzp + c0;
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              const float4 q = *reinterpret_cast<const float4*>(zp + j);
              h[j] = v[j] * gelu_grad(q.x);
              h[j + 1] = v[j + 1] * gelu_grad(q.y);
              h[j + 2] = v[j + 2] * gelu_grad(q.z);
              h[j + 3] = v[j + 3] * gelu_grad(q.w);
            }
          }
          // plain: eight consecutive columns are 16 contiguous bytes
          if (g.H) {
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
              uint4 pk;
              pk.x = pack_bf16x2(h[j], h[j + 1]);
              pk.y = pack_bf16x2(h[j + 2], h[j + 3]);
              pk.z = pack_bf16x2(h[j + 4], h[j + 5]);
              pk.w = pack_bf16x2(h[j + 6], h[j + 7]);
              *reinterpret_cast<uint4*>(g.H + tl_off(m, c0 + j, g.MA)) = pk;
            }
          }
          // transposed: element (column, row)
          if (g.HT) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              *reinterpret_cast<bf16*>(g.HT + tl_off(c0 + j, m, N)) = __float2bfloat16(h[j]);
          }
        }
      }
    }
  }
done:
  tc_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

template <int N>
constexpr size_t gemm_smem() {
  return (size_t)NSTAGE * (kAChunk + N * KCH * 2) + 16 * NSTAGE + 8 + 16 + 1024;
}

template <int N, int EPI>
cudaError_t launch_n(const TcGemmArgs& g, int mtiles, int splits, cudaStream_t s) {
  auto kern = tc_gemm_kernel<N, EPI>;
  const size_t sm = gemm_smem<N>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<dim3((unsigned)mtiles, (unsigned)splits), kThreads, sm, s>>>(g);
  return cudaGetLastError();
}

}  // namespace

cudaError_t tc_gemm(const TcGemmArgs& g, int n, int epi, int mtiles, int splits,
                    cudaStream_t s) {
  if (g.K % KCH || g.MA % TMR || mtiles < 1 || splits < 1 ||
      (int64_t)splits * g.kchunks_per_split < g.K / KCH ||
      (int64_t)(splits - 1) * g.kchunks_per_split >= g.K / KCH)
    return cudaErrorInvalidValue;  // every split must own at least one K-chunk
  switch (n * 8 + epi) {
    case 256 * 8 + EPI_HIDDEN: return launch_n<256, EPI_HIDDEN>(g, mtiles, splits, s);
    case 256 * 8 + EPI_DX: return launch_n<256, EPI_DX>(g, mtiles, splits, s);
    case 256 * 8 + EPI_PARTIAL: return launch_n<256, EPI_PARTIAL>(g, mtiles, splits, s);
    case 32 * 8 + EPI_PARTIAL: return launch_n<32, EPI_PARTIAL>(g, mtiles, splits, s);
    case 16 * 8 + EPI_OUT: return launch_n<16, EPI_OUT>(g, mtiles, splits, s);
    case 16 * 8 + EPI_PARTIAL: return launch_n<16, EPI_PARTIAL>(g, mtiles, splits, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nn
}  // namespace vfisv
