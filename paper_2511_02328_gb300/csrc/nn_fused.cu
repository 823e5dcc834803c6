// nn_fused.cu -- the classifier's inference in one kernel: one block per
// image, every activation in shared memory (the layered path of model.cu,
// which keeps the activations for the backward pass, serves training).
//
// Same network and precision policy: input bf16 [64][64][2]; three blocks
// conv3x3 (pad 1) + bias -> ReLU -> 2x2 max pool, 2 -> 16 -> 32 -> 64
// channels, the pooled activations rounded to bf16; global average pool,
// FC 64 -> 2, softmax.  Weights are rounded from the fp32 master parameters to
// bf16 (nearest even) in shared memory.
//
// Each convolution is an implicit GEMM on mma.sync.m16n8k16 (bf16 -> fp32):
// an M tile is a 2 x 8 pixel patch (rows g and g + 8 of the fragment are the
// vertically adjacent pixels (y, x) and (y + 1, x), x = 8 tx + g), so a 2x2
// pool window sits in one thread (vertical pair) and its neighbour lane
// g ^ 1 (horizontal pair, one shuffle); A fragments are read straight from
// the NHWC activations (a 32-bit word = two consecutive input channels of one
// tap, k = (dy * 3 + dx) * cin + i), B fragments from the packed weights
// [cout][K].  Bias, ReLU, pooling and the bf16 rounding happen in the
// accumulator registers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"
#include "nn.h"

namespace {

constexpr int FT = 256;          // threads (8 warps)
constexpr int NWF = FT / 32;

// shared-memory layout (bf16 elements unless noted)
constexpr int IN_E = 66 * 66 * 2;    // input with a 1-pixel zero halo
constexpr int A1_E = 34 * 34 * 16;   // block 1 output (pooled, halo)
constexpr int A2_E = 18 * 18 * 32;   // block 2 output (pooled, halo)
constexpr int A3_E = 8 * 8 * 64;     // block 3 output (pooled)
constexpr int K1 = 32, K2 = 144, K3 = 288;   // padded K of each conv (9 cin rounded up to 16)
constexpr int W1_E = 16 * K1, W2_E = 32 * K2, W3_E = 64 * K3;
constexpr int OFF_IN = 0, OFF_A1 = OFF_IN + IN_E, OFF_A2 = OFF_A1 + A1_E, OFF_A3 = OFF_A2 + A2_E;
constexpr int OFF_W1 = OFF_A3 + A3_E, OFF_W2 = OFF_W1 + W1_E, OFF_W3 = OFF_W2 + W2_E;
constexpr int BF_E = OFF_W3 + W3_E;                       // bf16 elements in total
constexpr int NF = 16 + 32 + 64 + 128 + 2 + 64 + 2;       // biases, fw, fb, gap, logits (floats)

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// conv3x3 + bias + ReLU + 2x2 max pool of one block.  in: [(H+2)][(H+2)][CIN]
// (zero halo), w: [COUT][KP], out: [(H/2 + 2 HALO)][...][COUT] (interior written).
template <int CIN, int COUT, int H, int KP, int HALO>
__device__ __forceinline__ void conv_block(const __nv_bfloat16* in, const __nv_bfloat16* w, const float* bias,
                                           __nv_bfloat16* out)
{
    constexpr int NT = COUT / 8, KS = KP / 16;
    constexpr int TX = H / 8, TILES = (H / 2) * TX;
    constexpr int OS = H / 2 + 2 * HALO;   // output row stride (pixels)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    for (int t = warp; t < TILES; t += NWF) {
        const int ty = t / TX, tx = t % TX;
        const int y0 = 2 * ty, x = 8 * tx + g;
        float acc[NT][4];
#pragma unroll
        for (int nt = 0; nt < NT; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) acc[nt][e] = 0.f;
#pragma unroll
        for (int ks = 0; ks < KS; ks++) {
            uint32_t a[4];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int kk = ks * 16 + 2 * q + 8 * h;
                const int pos = kk / CIN, i = kk % CIN;
                if (pos < 9) {
                    const int dy = pos / 3, dx = pos % 3;
                    a[2 * h] = ld32(in + ((y0 + dy) * (H + 2) + x + dx) * CIN + i);
                    a[2 * h + 1] = ld32(in + ((y0 + 1 + dy) * (H + 2) + x + dx) * CIN + i);
                } else {
                    a[2 * h] = a[2 * h + 1] = 0u;
                }
            }
#pragma unroll
            for (int nt = 0; nt < NT; nt++) {
                const __nv_bfloat16* wr = w + (nt * 8 + g) * KP + ks * 16 + 2 * q;
                mma_bf16(acc[nt], a, ld32(wr), ld32(wr + 8));
            }
        }
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            const int col = nt * 8 + 2 * q;
            float v0 = fmaxf(fmaxf(acc[nt][0] + bias[col], 0.f), fmaxf(acc[nt][2] + bias[col], 0.f));
            float v1 = fmaxf(fmaxf(acc[nt][1] + bias[col + 1], 0.f), fmaxf(acc[nt][3] + bias[col + 1], 0.f));
            v0 = fmaxf(v0, __shfl_xor_sync(0xffffffffu, v0, 4));
            v1 = fmaxf(v1, __shfl_xor_sync(0xffffffffu, v1, 4));
            if ((g & 1) == 0) {
                const int py = ty + HALO, px = (x >> 1) + HALO;
                *reinterpret_cast<__nv_bfloat162*>(out + (py * OS + px) * COUT + col) = __floats2bfloat162_rn(v0, v1);
            }
        }
    }
}

__global__ void __launch_bounds__(FT, 1)
k_forward_fused(const __nv_bfloat16* __restrict__ x, const float* __restrict__ w0, const float* __restrict__ b0,
                const float* __restrict__ w1, const float* __restrict__ b1, const float* __restrict__ w2,
                const float* __restrict__ b2, const float* __restrict__ fw, const float* __restrict__ fb,
                float* __restrict__ logits, float* __restrict__ prob)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __nv_bfloat16* S = reinterpret_cast<__nv_bfloat16*>(smem);
    float* F = reinterpret_cast<float*>(smem + (size_t)BF_E * 2);
    float *sb0 = F, *sb1 = F + 16, *sb2 = F + 48, *sfw = F + 112, *sfb = F + 240, *gap = F + 242, *lg = F + 306;
    const int tid = threadIdx.x;
    const int img = blockIdx.x;

    // zero the activation buffers (halos and padding), then fill input, weights, constants
    uint32_t* Z = reinterpret_cast<uint32_t*>(S);
    for (int i = tid; i < OFF_W1 / 2; i += FT) Z[i] = 0u;
    __syncthreads();
    const uint32_t* xi = reinterpret_cast<const uint32_t*>(x + (int64_t)img * 64 * 64 * 2);
    uint32_t* in = reinterpret_cast<uint32_t*>(S + OFF_IN);
    for (int p = tid; p < 64 * 64; p += FT) in[((p >> 6) + 1) * 66 + (p & 63) + 1] = __ldg(xi + p);
    for (int e = tid; e < W1_E; e += FT) {
        const int o = e / K1, k = e % K1;
        S[OFF_W1 + e] = __float2bfloat16_rn(k < 18 ? __ldg(w0 + o * 18 + k) : 0.f);
    }
    for (int e = tid; e < W2_E; e += FT) S[OFF_W2 + e] = __float2bfloat16_rn(__ldg(w1 + e));
    for (int e = tid; e < W3_E; e += FT) S[OFF_W3 + e] = __float2bfloat16_rn(__ldg(w2 + e));
    if (tid < 16) sb0[tid] = __ldg(b0 + tid);
    if (tid < 32) sb1[tid] = __ldg(b1 + tid);
    if (tid < 64) sb2[tid] = __ldg(b2 + tid);
    if (tid < 128) sfw[tid] = __ldg(fw + tid);
    if (tid < 2) sfb[tid] = __ldg(fb + tid);
    __syncthreads();

    conv_block<2, 16, 64, K1, 1>(S + OFF_IN, S + OFF_W1, sb0, S + OFF_A1);
    __syncthreads();
    conv_block<16, 32, 32, K2, 1>(S + OFF_A1, S + OFF_W2, sb1, S + OFF_A2);
    __syncthreads();
    conv_block<32, 64, 16, K3, 0>(S + OFF_A2, S + OFF_W3, sb2, S + OFF_A3);
    __syncthreads();

    // global average pool (fixed order), FC, softmax
    if (tid < 64) {
        float acc = 0.f;
        for (int p = 0; p < 64; p++) acc += __bfloat162float(S[OFF_A3 + p * 64 + tid]);
        gap[tid] = acc / 64.f;
    }
    __syncthreads();
    if (tid < 2) {
        float v = sfb[tid];
        for (int i = 0; i < 64; i++) v += gap[i] * sfw[tid * 64 + i];
        lg[tid] = v;
    }
    __syncthreads();
    if (tid == 0) {
        const float mx = fmaxf(lg[0], lg[1]);
        const float e0 = expf(lg[0] - mx), e1 = expf(lg[1] - mx);
        logits[2 * img] = lg[0];
        logits[2 * img + 1] = lg[1];
        if (prob) prob[img] = e1 / (e0 + e1);
    }
}

}  // namespace

size_t nn_forward_fused_smem() { return (size_t)BF_E * 2 + (size_t)NF * 4; }

int nn_forward_fused(const __nv_bfloat16* x, int n, const float* w0, const float* b0, const float* w1,
                     const float* b1, const float* w2, const float* b2, const float* fw, const float* fb,
                     float* logits, float* prob, cudaStream_t s)
{
    if (n <= 0) return AF_OK;
    const size_t smem = nn_forward_fused_smem();
    if (int rc = af_ensure_smem((const void*)k_forward_fused, smem)) return rc;
    k_forward_fused<<<n, FT, smem, s>>>(x, w0, b0, w1, b1, w2, b2, fw, fb, logits, prob);
    return af_cuda_check(cudaGetLastError(), "fused forward launch");
}
