// Shapes, parameter-blob layout and host entry points of the initial-guess
// network (nn.cu) and of the mixed NN-initialised inversion (mixed.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "vfisv.h"

namespace vfisv {
namespace nn {

constexpr int IN = VFISV_NN_NIN, HID = VFISV_NN_NHID, OUT = VFISV_NN_NOUT;
constexpr int K0P = 64;      // input width padded for the tensor-core tiles
constexpr int N3P = 64;      // output width padded likewise
constexpr int kSplits = 32;  // most split-K CTAs per tile of the weight-gradient products

constexpr size_t OFF_W0 = 0;
constexpr size_t OFF_B0 = OFF_W0 + (size_t)IN * HID;
constexpr size_t OFF_W1 = OFF_B0 + HID;
constexpr size_t OFF_B1 = OFF_W1 + (size_t)HID * HID;
constexpr size_t OFF_W2 = OFF_B1 + HID;
constexpr size_t OFF_B2 = OFF_W2 + (size_t)HID * HID;
constexpr size_t OFF_W3 = OFF_B2 + HID;
constexpr size_t OFF_B3 = OFF_W3 + (size_t)HID * OUT;
constexpr size_t OFF_INM = OFF_B3 + OUT;
constexpr size_t OFF_INS = OFF_INM + IN;
constexpr size_t OFF_OUTM = OFF_INS + IN;
constexpr size_t OFF_OUTS = OFF_OUTM + (OUT - 1);
constexpr size_t NBLOB = OFF_OUTS + (OUT - 1);
constexpr size_t NTRAIN = OFF_INM;  // weights and biases (trained)
static_assert(NBLOB == VFISV_NN_NBLOB, "blob layout");

struct LayerDim {
  int K, N, Kp, Np;
  size_t offW, offB;
};
constexpr LayerDim kLayersHost[4] = {{IN, HID, K0P, HID, OFF_W0, OFF_B0},
                                     {HID, HID, HID, HID, OFF_W1, OFF_B1},
                                     {HID, HID, HID, HID, OFF_W2, OFF_B2},
                                     {HID, OUT, HID, N3P, OFF_W3, OFF_B3}};

// Affine permutation of sample indices: sample(m) = (mult (offset + m) + add) mod n.
struct Perm {
  uint64_t mult, add;
  int64_t offset, n;
};

// BF16 weight copies in the tiled layout of the training products (nn_tc.cuh)
struct PackedNet {
  uint8_t* Wt[4];  // element (output, input): forward B operand
  uint8_t* Wn[4];  // element (input, output): input-gradient B operand (layers 1-3)
};

size_t workspace_bytes(int64_t rows);
cudaError_t nn_init(void* ws, float* blob, const float* obs, const float* params, int64_t n,
                    uint64_t seed, cudaStream_t s);
cudaError_t nn_grad(void* ws, const float* blob, const float* obs, const float* params,
                    int64_t n, float* grad_out, float* loss_out, cudaStream_t s);
cudaError_t nn_train(void* ws, float* blob, const float* obs, const float* params, int64_t n,
                     int batch, int epochs, float lr0, uint64_t seed, float* loss_hist,
                     cudaStream_t s);
// Inference (mlp_tc.cu): one fused tensor-core kernel from observations to
// initial models.  The workspace holds the device error word (first
// kNnErrBytes) and the packed BF16 weights (kTcPackBytes after it).
constexpr size_t kNnErrBytes = 256;
constexpr size_t kTcPackBytes = 286720;
constexpr size_t infer_workspace_bytes() { return kNnErrBytes + kTcPackBytes; }
cudaError_t nn_infer(void* ws, const float* blob, const float* obs, int64_t n, float mu,
                     float* init, float* conf, float* raw, cudaStream_t s);
// rows the gradient/forward paths pad a batch of n samples to
int64_t padded_rows(int64_t n);

// mixed.cu: route by the confidence output (the listed pixels run LM from
// the guess; the others get an empty first-stage result), flag pixels for
// plain re-inversion, gather them, merge results.
cudaError_t route_by_confidence(const float* conf, int64_t npix, float conf_route,
                                const float* init, int64_t* list, int64_t* count, float* params,
                                float* chi2, int32_t* iters, int32_t* status, cudaStream_t s);
cudaError_t flag_and_gather(const int32_t* status, const float* chi2, int64_t npix,
                            float chi2_flag, bool flag_unconverged, const float* obs, const float* w,
                            int64_t w_stride, int nobs, int64_t* count, int64_t* index,
                            float* obs_g, float* w_g, int32_t* flagged, cudaStream_t s);
cudaError_t merge_plain(const int64_t* count, const int64_t* index, int64_t npix_max,
                        const float* p2, const float* c2, const int32_t* i2, const int32_t* s2,
                        const float* cov2, float* params, float* chi2, int32_t* iters,
                        int32_t* status, float* cov, cudaStream_t s);

}  // namespace nn
}  // namespace vfisv
