// nn.h -- internal declarations of the classifier kernels (nn.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "afgb.h"

// GEMM operand layouts: A K-major ([M][K]) or M-major ([K][M]); B K-major
// ([N][K]) or N-major ([K][N]).
enum { NN_A_K_B_K = 0, NN_A_K_B_N = 1, NN_A_M_B_N = 2, NN_A_M_B_K = 3 };
// Epilogues: store fp32; add bias[n] then ReLU, store fp32; atomic add fp32 (split-K).
enum { NN_EPI_STORE = 0, NN_EPI_BIAS_RELU = 1, NN_EPI_ATOMIC = 2 };

// Plain GEMM on the tensor cores (conv_umma.cu); a bounded wait that runs out
// raises *err.
int nn_gemm(int layout, int epi, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
            int splits, float* C, int ldc, const float* bias, int* err, cudaStream_t s);
// 3x3 convolutions (pad 1) of classifier layer 0, 1, 2 (2 -> 16 -> 32 -> 64
// channels, 64 / 32 / 16 pixels square) on the tensor cores with TMA-staged
// operands (conv_tma.cu).  Tensors are channel-blocked, [n][C/8][H][W][8]
// bf16 (the first layer's input: the raw [n][64][64][2], which the layer-0
// kernels expand in shared memory to 8 channels, those of columns x - 1, x,
// x + 1 and two zeros):
//   forward: x -> bias, ReLU, 2x2 max pool -> out [n][cout/8][H/2][W/2][8] and
//            idx (argmax 0..3 | 4 if positive, laid out as out; nullable)
//   dgrad:   dz [n][cout/8][H][W][8] -> dx [n][cin/8][H][W][8] (layers 1, 2)
//   wgrad:   grad [cout][9][cin] += sum_p dz[p] (x) x[p + tap]
// Weights come packed by nn_tpack (nn_tpack_bytes bytes; dgrad != 0: the
// data gradient's transposed, flipped form).  A bounded wait that runs out
// raises *err.
int nn_tconv_fwd(int layer, const __nv_bfloat16* x, int n, const __nv_bfloat16* wp, const float* bias,
                 __nv_bfloat16* out, uint8_t* idx, int* err, cudaStream_t s);
int nn_tconv_dgrad(int layer, const __nv_bfloat16* dz, int n, const __nv_bfloat16* wp, __nv_bfloat16* dx, int* err,
                   cudaStream_t s);
int nn_tconv_wgrad(int layer, const __nv_bfloat16* dz, const __nv_bfloat16* x, int n, float* grad, int* err,
                   cudaStream_t s);
// Layer 0's weight gradient straight from the pooled gradient dp [n][2][32][32][8]
// and the argmax bytes idx (laid out as dp): the 2x2 max-pool backward pass
// runs inside it (dz is never stored), and the bias gradient (the sum of dz)
// is added to db [16].
int nn_tconv_wgrad_unpool(const __nv_bfloat16* dp, const uint8_t* idx, const __nv_bfloat16* x, int n, float* grad,
                          float* db, int* err, cudaStream_t s);
size_t nn_tpack_bytes(int layer, int dgrad);
int nn_tpack(int layer, int dgrad, const float* w, __nv_bfloat16* out, cudaStream_t s);
// 2x2 max-pool backward on channel-blocked tensors (dz [n][c/8][H][W][8] from
// the pooled gradient and the argmax bytes, both [n][c/8][H/2][W/2][8]); adds
// the bias gradient (sum of dz over pixels) into db.
int nn_pool_back(const __nv_bfloat16* dp, const uint8_t* idx, int n, int H, int W, int c, __nv_bfloat16* dz,
                 float* db, cudaStream_t s);
int nn_head(const __nv_bfloat16* a3, int n, const float* fw, const float* fb, float* logits, float* prob,
            const int32_t* y, float* loss, float* dfw, float* dfb, __nv_bfloat16* da3, cudaStream_t s);
int nn_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, int step, cudaStream_t s);
int nn_f32_to_bf16(const float* x, int64_t n, __nv_bfloat16* y, cudaStream_t s);
int nn_cutouts(const uint8_t* X, int64_t nsamp, int nchan, const int32_t* D, int ndm, const int32_t* plane,
               int64_t nout, const af_cand_t* cands, int n, __nv_bfloat16* out, cudaStream_t s);
// Inference in one kernel (nn_fused.cu): logits [n][2] and P(pulse) [n] of
// bf16 inputs [n][64][64][2]; weights from the fp32 master parameters.
size_t nn_forward_fused_smem();
int nn_forward_fused(const __nv_bfloat16* x, int n, const float* w0, const float* b0, const float* w1,
                     const float* b1, const float* w2, const float* b2, const float* fw, const float* fb,
                     float* logits, float* prob, cudaStream_t s);
