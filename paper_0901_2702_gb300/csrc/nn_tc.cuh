// The tcgen05 training GEMM (nn_tc.cu) and its operand layout, used by the
// network's forward and backward passes (nn.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vfisv {
namespace nn {

// Byte offset of element (r, c) of an R x C BF16 matrix in the tiled
// canonical layout TL(R, C): 64-column chunks one after the other (R * 128
// bytes each), 8-row groups of 1024 bytes, 128-byte core matrices of 8 rows
// x 8 columns along K.
__host__ __device__ constexpr size_t tl_off(int64_t r, int c, int64_t R) {
  return (size_t)(c >> 6) * (size_t)R * 128 + (size_t)(r >> 3) * 1024 +
         (size_t)((c & 63) >> 3) * 128 + (size_t)(r & 7) * 16 + (size_t)(c & 7) * 2;
}

// Epilogues of D = A B^T (rows of D = rows of A).
enum TcEpi : int {
  EPI_HIDDEN = 0,   // z = D + bias -> Z (FP32, row-major); GELU(z) -> H, HT (BF16, TL)
  EPI_OUT = 1,      // D + bias (first n_valid columns) -> Z (FP32, row-major)
  EPI_DX = 2,       // D * GELU'(Zprev) -> H, HT (BF16, TL); H may be null
  EPI_PARTIAL = 3,  // D of this K split -> P[split][MA][N] (FP32)
};

struct TcGemmArgs {
  const uint8_t* A;  // TL(MA, K)
  int64_t MA;        // rows of A (a multiple of 128) = rows of D
  const uint8_t* B;  // TL(NB, K), NB = N
  int64_t NB;
  int K;                  // a multiple of 64
  int kchunks_per_split;  // 64-wide K-chunks per blockIdx.y
  const float* bias;
  int n_valid;
  float* Z;
  int64_t ldz;
  uint8_t* H;   // TL(MA, N)
  uint8_t* HT;  // TL(N, MA)
  const float* Zprev;
  int64_t ldzp;
  float* P;
  int* err;
};

// D tiles of N in {16, 32, 256} columns; grid mtiles x splits.  Returns
// cudaErrorInvalidValue for shapes the kernel does not take (K or MA not
// multiples of 64 / 128, a split without K-chunks, an unsupported N/epilogue).
cudaError_t tc_gemm(const TcGemmArgs& g, int n, int epi, int mtiles, int splits, cudaStream_t s);

}  // namespace nn
}  // namespace vfisv
