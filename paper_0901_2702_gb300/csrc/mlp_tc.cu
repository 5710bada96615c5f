// Inference of the initial-guess network (Sec. 5) on the fifth-generation
// tensor cores, fused end to end: one persistent kernel takes a tile of 128
// pixels from the observed Stokes samples through the input features, the
// four layers and the decoding into an initial model.  Every layer is a chain
// of tcgen05.mma (M = 128, K = 16 per instruction, BF16 operands in shared
// memory, FP32 accumulators in tensor memory); the bias + GELU epilogues read
// the accumulators back with tcgen05.ld, 16 warps each owning a lane quarter
// and a column quarter, and write the next layer's BF16 operand to shared
// memory.  Nothing but the observations and the outputs touches HBM.
//
// Shared-memory operands are in the no-swizzle K-major canonical layout of
// the MMA descriptors: core matrices of 8 rows x 16 bytes stored as 128
// contiguous bytes, core matrices adjacent along K 128 bytes apart (the
// leading-dimension offset) and 8-row groups `sbo` bytes apart (the
// stride-dimension offset).  The hidden layers' weights (2 x 128 KB) do not
// fit beside the 64 KB activation tile, so they stream through a three-slot
// ring of 32 KB K-chunks filled by bulk copies (the same 256 KB per tile,
// served from L2); W0 (16 KB) and W3 (8 KB) stay resident.
//
// Every wait is bounded (about 1 s); on a timeout the kernel lets its copies
// and tensor-core work in flight finish (bounded again), frees its tensor
// memory, writes kDevErrNnWait to the error word and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"
#include "nn.cuh"
#include "nn_device.cuh"
#include "tc_device.cuh"

namespace vfisv {
namespace nn {

namespace {

using bf16 = __nv_bfloat16;

constexpr int TM = 128;       // pixels per tile = MMA M
constexpr int K0 = 32;        // input width (24) padded to two K = 16 steps
constexpr int N3 = 16;        // output width (11) padded to the smallest N for M = 128
constexpr int KC = 64;        // K-chunk of a streamed hidden-layer weight block
constexpr int NSLOT = 3;      // weight ring depth
constexpr int THREADS = 512;  // 16 warps: 4 lane quarters x 4 column quarters
constexpr int kChunks = HID / KC;           // chunks per hidden layer
constexpr int kStreamPerTile = 2 * kChunks; // streamed chunks per tile (W1, W2)

constexpr uint32_t kChunkBytes = HID * KC * 2;    // 32768
constexpr uint32_t kW0Bytes = HID * K0 * 2;       // 16384
constexpr uint32_t kLayerBytes = HID * HID * 2;   // 131072
constexpr uint32_t kW3Bytes = N3 * HID * 2;       // 8192
constexpr uint32_t kHChunkBytes = TM * KC * 2;    // 16384: one K-chunk of the activations
constexpr uint32_t kW3ChunkBytes = N3 * KC * 2;   // 2048
static_assert(kW0Bytes + 2 * kLayerBytes + kW3Bytes == kTcPackBytes, "packed weight size");

// Shared-memory carve, bytes from a 1024-byte aligned base.
constexpr uint32_t SM_RING = 0;
constexpr uint32_t SM_H = SM_RING + NSLOT * kChunkBytes;
constexpr uint32_t SM_W0 = SM_H + TM * HID * 2;
constexpr uint32_t SM_W3 = SM_W0 + kW0Bytes;
constexpr uint32_t SM_X = SM_W3 + kW3Bytes;
constexpr uint32_t SM_BIAS = SM_X + TM * K0 * 2;          // b0 | b1 | b2 | b3 (16)
constexpr uint32_t SM_STAT = SM_BIAS + (3 * HID + N3) * 4;  // in_mean 24 | in_std 24 | out_mean 16 | out_std 16
constexpr uint32_t SM_BAR = SM_STAT + 80 * 4;             // full[3] empty[3] weights mma
constexpr uint32_t SM_TMEM = SM_BAR + 8 * 8;
constexpr uint32_t SM_END = SM_TMEM + 16;
constexpr size_t kSmemBytes = SM_END + 1024;
static_assert(SM_BAR % 8 == 0, "mbarrier alignment");
static_assert(kSmemBytes <= 232448, "shared memory per block");

constexpr int kTmemCols = 256;  // one M = 128 x N = 256 FP32 accumulator

constexpr uint32_t kIdescHid = idesc_bf16(TM, HID);
constexpr uint32_t kIdescOut = idesc_bf16(TM, N3);

// Packed weights (global, kTcPackBytes): W0 as one N = 256 x K = 32 block,
// W1 and W2 as four N = 256 x K = 64 chunks each, W3 as four N = 16 x K = 64
// chunks; element (n, k) is the weight from input k to output n, BF16,
// zero-padded.
__global__ void tc_pack_kernel(const float* __restrict__ blob, uint8_t* __restrict__ wp) {
  constexpr int E0 = HID * K0, E1 = HID * HID, E3 = N3 * HID;
  constexpr uint32_t sbo_w0 = (K0 / 8) * 128, sbo_c = (KC / 8) * 128;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < E0 + 2 * E1 + E3;
       i += gridDim.x * blockDim.x) {
    float w;
    uint32_t off;
    if (i < E0) {
      const int n = i / K0, k = i % K0;
      w = k < IN ? blob[OFF_W0 + (size_t)k * HID + n] : 0.0f;
      off = cm_off(n, k, sbo_w0);
    } else if (i < E0 + 2 * E1) {
      const int j = i - E0, l = j / E1, n = (j % E1) / HID, k = j % HID;
      w = blob[(l ? OFF_W2 : OFF_W1) + (size_t)k * HID + n];
      off = kW0Bytes + l * kLayerBytes + (k / KC) * kChunkBytes + cm_off(n, k % KC, sbo_c);
    } else {
      const int j = i - E0 - 2 * E1, n = j / HID, k = j % HID;
      w = n < OUT ? blob[OFF_W3 + (size_t)k * OUT + n] : 0.0f;
      off = kW0Bytes + 2 * kLayerBytes + (k / KC) * kW3ChunkBytes + cm_off(n, k % KC, sbo_c);
    }
    *reinterpret_cast<bf16*>(wp + off) = __float2bfloat16(w);
  }
}

struct TcArgs {
  const float* obs;  // [n][24]
  int64_t n;
  const float* blob;
  const uint8_t* wp;  // packed weights
  float mu;
  float* init;  // [n][10]
  float* conf;  // [n] or null
  float* raw;   // [n][11] or null
  int* err;
};

__global__ void __launch_bounds__(THREADS, 1) mlp_tc_kernel(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sb = smem_u32(sm);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* bias = reinterpret_cast<float*>(sm + SM_BIAS);
  float* stat = reinterpret_cast<float*>(sm + SM_STAT);
  const uint32_t bar_full = sb + SM_BAR, bar_empty = bar_full + 8 * NSLOT,
                 bar_w = bar_empty + 8 * NSLOT, bar_mma = bar_w + 8;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + SM_TMEM);

  const int64_t ntiles = (a.n + TM - 1) / TM;
  const int my_tiles = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
  const int total = my_tiles * kStreamPerTile;  // weight chunks this CTA streams

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 2 * NSLOT + 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_full + 8 * i), "r"(1)
                   : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < 3 * HID; i += THREADS) {
    const int l = i / HID;
    bias[i] = a.blob[(l == 0 ? OFF_B0 : l == 1 ? OFF_B1 : OFF_B2) + i % HID];
  }
  if (tid < N3) bias[3 * HID + tid] = tid < OUT ? a.blob[OFF_B3 + tid] : 0.0f;
  if (tid < IN) {
    stat[tid] = a.blob[OFF_INM + tid];
    stat[IN + tid] = a.blob[OFF_INS + tid];
  }
  if (tid < OUT - 1) {
    stat[48 + tid] = a.blob[OFF_OUTM + tid];
    stat[64 + tid] = a.blob[OFF_OUTS + tid];
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = *tmem_slot;

  // issuer state (thread 0): stream cursors and a sticky timeout flag
  int g_cons = 0, g_load = 0, g_landed = 0;
  bool ibad = false, w_landed = false;
  auto load_chunk = [&](int g) {
    const int slot = g % NSLOT, q = g % kStreamPerTile;
    const uint8_t* src = a.wp + kW0Bytes + (q / kChunks) * kLayerBytes + (q % kChunks) * kChunkBytes;
    expect_tx(bar_full + 8 * slot, kChunkBytes);
    bulk_load(sb + SM_RING + slot * kChunkBytes, src, kChunkBytes, bar_full + 8 * slot);
  };
  if (tid == 0) {
    expect_tx(bar_w, kW0Bytes + kW3Bytes);
    bulk_load(sb + SM_W0, a.wp, kW0Bytes, bar_w);
    bulk_load(sb + SM_W3, a.wp + kW0Bytes + 2 * kLayerBytes, kW3Bytes, bar_w);
    for (; g_load < 2 && g_load < total; ++g_load) load_chunk(g_load);
  }

  // one hidden layer from the streamed chunks: D = H W^T, K = 256
  auto issue_hidden = [&]() {
    tc_after_sync();
    for (int c = 0; c < kChunks; ++c) {
      const int g = g_cons++;
      const int slot = g % NSLOT;
      if (!ibad) {
        if (mbar_wait(bar_full + 8 * slot, (g / NSLOT) & 1)) {
          g_landed = g + 1;
#pragma unroll
          for (int ks = 0; ks < KC / 16; ++ks)
            mma_bf16(tmem, sdesc(sb + SM_H + c * kHChunkBytes + ks * 256, 128, 1024),
                     sdesc(sb + SM_RING + slot * kChunkBytes + ks * 256, 128, 1024), kIdescHid,
                     (c | ks) != 0);
          mma_commit(bar_empty + 8 * slot);
        } else {
          ibad = true;
        }
      }
      // refill the slot of chunk g - 1 (its MMAs were issued earlier) with g + 2
      const int gn = g + 2;
      if (!ibad && gn < total) {
        if (gn >= NSLOT && !mbar_wait(bar_empty + 8 * (gn % NSLOT), (gn / NSLOT - 1) & 1)) {
          ibad = true;
        } else {
          load_chunk(gn);
          g_load = gn + 1;
        }
      }
    }
    mma_commit(bar_mma);
  };

  uint32_t mph = 0;
  // every thread waits for the layer's MMAs; the CTA continues only if none
  // timed out (and the issuer saw no timeout)
  auto sync_mma = [&]() -> bool {
    const bool ok = mbar_wait(bar_mma, mph);
    mph ^= 1;
    if (__syncthreads_or(!ok || (tid == 0 && ibad))) return false;
    tc_after_sync();
    return true;
  };

  // bias + GELU of the accumulator -> BF16 activations (next layer's A)
  auto epilogue_hidden = [&](const float* b) {
    const int q = warp & 3, cq = warp >> 2, row = 32 * q + lane;
    uint8_t* hrow = sm + SM_H + cq * kHChunkBytes + (row >> 3) * 1024 + (row & 7) * 16;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int col0 = cq * KC + 32 * half;
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col0, v);
#pragma unroll
      for (int g8 = 0; g8 < 4; ++g8) {
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 8 * g8 + 2 * e;
          pk[e] = pack_bf16x2(gelu(v[j] + b[col0 + j]), gelu(v[j + 1] + b[col0 + j + 1]));
        }
        *reinterpret_cast<uint4*>(hrow + (4 * half + g8) * 128) =
            make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
  };

  bool ok = true;
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    // features: thread (row, part) writes input columns 8 part .. 8 part + 7
    float ic_row = 1.0f;
    {
      const int row = tid & (TM - 1), part = tid >> 7;
      const int64_t m = tile * TM + row;
      uint32_t pk[4] = {0u, 0u, 0u, 0u};
      if (m < a.n) {
        const float* o = a.obs + m * IN;
        ic_row = ic_of(o);
        if (part < IN / 8) {
          const float inv = 1.0f / ic_row;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int j = 8 * part + 2 * e;
            pk[e] = pack_bf16x2((o[j] * inv - stat[j]) / stat[IN + j],
                                (o[j + 1] * inv - stat[j + 1]) / stat[IN + j + 1]);
          }
        }
      }
      *reinterpret_cast<uint4*>(sm + SM_X + cm_off(row, 8 * part, (K0 / 8) * 128)) =
          make_uint4(pk[0], pk[1], pk[2], pk[3]);
      fence_async_smem();
      tc_before_sync();
      __syncthreads();
    }
    // layer 0: K = 32 from X and the resident W0
    if (tid == 0) {
      tc_after_sync();
      if (!w_landed && !ibad) {
        if (mbar_wait(bar_w, 0)) w_landed = true;
        else ibad = true;
      }
      if (!ibad)
#pragma unroll
        for (int ks = 0; ks < K0 / 16; ++ks)
          mma_bf16(tmem, sdesc(sb + SM_X + ks * 256, 128, (K0 / 8) * 128),
                   sdesc(sb + SM_W0 + ks * 256, 128, (K0 / 8) * 128), kIdescHid, ks != 0);
      mma_commit(bar_mma);
    }
    if (!(ok = sync_mma())) break;
    epilogue_hidden(bias);
    // layers 1 and 2 from the streamed chunks
    if (tid == 0) issue_hidden();
    if (!(ok = sync_mma())) break;
    epilogue_hidden(bias + HID);
    if (tid == 0) issue_hidden();
    if (!(ok = sync_mma())) break;
    epilogue_hidden(bias + 2 * HID);
    // output layer: N = 16 from the resident W3
    if (tid == 0) {
      tc_after_sync();
      if (!ibad)
        for (int c = 0; c < kChunks; ++c)
#pragma unroll
          for (int ks = 0; ks < KC / 16; ++ks)
            mma_bf16(tmem, sdesc(sb + SM_H + c * kHChunkBytes + ks * 256, 128, 1024),
                     sdesc(sb + SM_W3 + c * kW3ChunkBytes + ks * 256, 128, 1024), kIdescOut,
                     (c | ks) != 0);
      mma_commit(bar_mma);
    }
    if (!(ok = sync_mma())) break;
    if (warp < 4) {  // lane quarter `warp`, row = tid
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16), v);
      const int64_t m = tile * TM + tid;
      if (m < a.n) {
        float y[OUT];
#pragma unroll
        for (int o = 0; o < OUT; ++o) y[o] = v[o] + bias[3 * HID + o];
        decode_row(y, ic_row, a.mu, stat + 48, stat + 64, a.init + m * 10);
        if (a.conf) a.conf[m] = y[OUT - 1];
        if (a.raw)
#pragma unroll
          for (int o = 0; o < OUT; ++o) a.raw[m * OUT + o] = y[o];
      }
    }
    tc_before_sync();
  }

  if (ok && tid == 0) {
    // the tensor cores' last arrivals on the slot barriers precede the exit
    for (int g = total > NSLOT ? total - NSLOT : 0; g < total; ++g)
      mbar_wait(bar_empty + 8 * (g % NSLOT), (g / NSLOT) & 1);
  }
  if (!ok && tid == 0) {
    // let the tensor-core work and the copies in flight land before the
    // shared and tensor memory are released
    mbar_wait(bar_mma, mph ^ 1);
    for (int g = g_landed; g < g_load; ++g) mbar_wait(bar_full + 8 * (g % NSLOT), (g / NSLOT) & 1);
    if (!w_landed) mbar_wait(bar_w, 0);
    atomicExch(a.err, kDevErrNnWait);
  }
  tc_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

}  // namespace

cudaError_t nn_infer(void* ws, const float* blob, const float* obs, int64_t n, float mu,
                     float* init, float* conf, float* raw, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  uint8_t* wp = static_cast<uint8_t*>(ws) + kNnErrBytes;
  tc_pack_kernel<<<140, 256, 0, s>>>(blob, wp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  nsm = sm_budget(nsm);
  if ((e = cudaFuncSetAttribute(mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmemBytes)) != cudaSuccess)
    return e;
  const int64_t ntiles = (n + TM - 1) / TM;
  TcArgs a{obs, n, blob, wp, mu, init, conf, raw, static_cast<int*>(ws)};
  mlp_tc_kernel<<<(unsigned)(ntiles < nsm ? ntiles : nsm), THREADS, kSmemBytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace nn
}  // namespace vfisv
