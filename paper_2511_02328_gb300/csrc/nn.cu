// nn.cu -- elementwise and reduction kernels of the candidate classifier
// (replaces the paper's YOLO detector, Sec. 2.5): the 2x2 max-pool backward
// pass, the bias gradient, the classifier head (global average pool, fully
// connected layer, softmax cross-entropy) and Adam, on the channel-blocked
// activations of the tensor-core convolutions (conv_tma.cu).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "nn.h"

namespace {

// dz [n][C/8][H][W][8] (bf16) = the pooled gradient dp [n][C/8][H/2][W/2][8]
// routed to the argmax of each 2x2 window where that maximum (a ReLU output)
// was positive: idx, laid out as dp, holds the argmax (0..3, raster order) |
// 4 when the maximum was > 0.  Thread = (pooled pixel, channel block): one
// 16-byte load of the gradient, one 8-byte load of the argmax bytes, four
// 16-byte stores.  Warp w of the grid keeps channel block w % CB and takes
// 32-pixel runs of every image (CB divides a block's 8 warps), so each
// thread's bias-gradient sums (the sums of dz) stay in registers: reduced per
// warp, then per block in shared memory, one atomic per channel and block.
__global__ void __launch_bounds__(256) k_pool_back(const __nv_bfloat16* __restrict__ dp, const uint8_t* __restrict__ idx,
                                                   int n, int H, int W, int CB, __nv_bfloat16* __restrict__ dz,
                                                   float* __restrict__ db)
{
    __shared__ float part[8][8];
    const int Ho = H / 2, Wo = W / 2, P = Ho * Wo, lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * 8 + wib, nw = (int64_t)gridDim.x * 8;
    const int cb = (int)(gw % CB);
    const int64_t total = (int64_t)n * P;  // (image, pooled pixel) pairs
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t f = (gw / CB) * 32 + lane; f < total; f += (nw / CB) * 32) {
        const int64_t img = f / P;
        const int p = (int)(f - img * P), yo = p / Wo, xo = p - yo * Wo;
        const int64_t e = ((img * CB + cb) * P + p) * 8;
        const uint4 v = *reinterpret_cast<const uint4*>(dp + e);
        const uint2 ix = *reinterpret_cast<const uint2*>(idx + e);
        const uint16_t* vv = reinterpret_cast<const uint16_t*>(&v);
        const uint8_t* ii = reinterpret_cast<const uint8_t*>(&ix);
#pragma unroll
        for (int j = 0; j < 8; j++)
            if (ii[j] & 4) acc[j] += __bfloat162float(__ushort_as_bfloat16(vv[j]));
        __nv_bfloat16* zp = dz + (img * CB + cb) * (int64_t)H * W * 8;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t lo = ii[2 * j] == (uint8_t)(4 | q) ? vv[2 * j] : 0u;
                const uint32_t hi = ii[2 * j + 1] == (uint8_t)(4 | q) ? vv[2 * j + 1] : 0u;
                w[j] = lo | (hi << 16);
            }
            const int y = 2 * yo + (q >> 1), x = 2 * xo + (q & 1);
            *reinterpret_cast<uint4*>(zp + ((int64_t)y * W + x) * 8) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
#pragma unroll
    for (int j = 0; j < 8; j++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
        if (lane == 0) part[wib][j] = acc[j];
    }
    __syncthreads();
    if ((int)threadIdx.x < 8 * CB) {
        // channel 8 c + j is summed by the warps whose block is c
        const int c = threadIdx.x / 8, j = threadIdx.x % 8;
        float sum = 0.f;
        for (int w = c; w < 8; w += CB) sum += part[w][j];
        atomicAdd(db + threadIdx.x, sum);
    }
}

// Head: per sample, global average pool of a3 [n][8][64 positions][8] (bf16,
// channel-blocked: channel c at block c / 8, lane c % 8),
// logits = g fw^T + fb, softmax; with labels, the mean cross-entropy and its
// gradients (dfw, dfb accumulated, da3 written as bf16).
__global__ void k_head(const __nv_bfloat16* __restrict__ a3, int n, const float* __restrict__ fw,
                       const float* __restrict__ fb, float* __restrict__ logits, float* __restrict__ prob,
                       const int32_t* __restrict__ y, float* __restrict__ loss, float* __restrict__ dfw,
                       float* __restrict__ dfb, __nv_bfloat16* __restrict__ da3)
{
    const int s = blockIdx.x;
    const int ch = threadIdx.x;  // 64 threads
    __shared__ float g[64], lg[2];
    const __nv_bfloat16* a = a3 + ((int64_t)s * 8 + ch / 8) * 64 * 8 + ch % 8;
    float acc = 0.f;
    for (int q = 0; q < 64; q++) acc += __bfloat162float(a[q * 8]);
    g[ch] = acc / 64.f;
    __syncthreads();
    if (ch < 2) {
        float v = fb[ch];
        for (int i = 0; i < 64; i++) v += g[i] * fw[ch * 64 + i];
        lg[ch] = v;
    }
    __syncthreads();
    const float mx = fmaxf(lg[0], lg[1]);
    const float e0 = expf(lg[0] - mx), e1 = expf(lg[1] - mx);
    const float p0 = e0 / (e0 + e1), p1 = e1 / (e0 + e1);
    if (ch == 0) {
        logits[2 * s] = lg[0];
        logits[2 * s + 1] = lg[1];
        if (prob) prob[s] = p1;
    }
    if (!y) return;
    const int lab = y[s];
    const float inv = 1.f / (float)n;
    const float d0 = (p0 - (lab == 0 ? 1.f : 0.f)) * inv, d1 = (p1 - (lab == 1 ? 1.f : 0.f)) * inv;
    if (ch == 0) {
        atomicAdd(loss, -logf(lab == 1 ? p1 : p0) * inv);
        atomicAdd(dfb, d0);
        atomicAdd(dfb + 1, d1);
    }
    atomicAdd(dfw + ch, d0 * g[ch]);
    atomicAdd(dfw + 64 + ch, d1 * g[ch]);
    const float dg = (d0 * fw[ch] + d1 * fw[64 + ch]) / 64.f;
    const __nv_bfloat16 v = __float2bfloat16(dg);
    __nv_bfloat16* d = da3 + ((int64_t)s * 8 + ch / 8) * 64 * 8 + ch % 8;
    for (int q = 0; q < 64; q++) d[q * 8] = v;
}

// Adam on fp32 master weights (Kingma & Ba 2015, bias-corrected).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_f32_to_bf16(const float* __restrict__ x, int64_t n, __nv_bfloat16* __restrict__ y)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

unsigned grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

int nn_pool_back(const __nv_bfloat16* dp, const uint8_t* idx, int n, int H, int W, int c, __nv_bfloat16* dz,
                 float* db, cudaStream_t s)
{
    const int CB = c / 8;
    if (c % 8 || (CB != 1 && CB != 2 && CB != 4 && CB != 8) || ((uintptr_t)dp & 15) || ((uintptr_t)dz & 15) ||
        ((uintptr_t)idx & 7))
        return af_set_error(AF_EINVAL, "pool backward: channels / alignment");
    const int64_t warps = CB * (((int64_t)n * (H / 2) * (W / 2) + 31) / 32);
    k_pool_back<<<grid_for(warps * 32, 256), 256, 0, s>>>(dp, idx, n, H, W, CB, dz, db);
    return af_cuda_check(cudaGetLastError(), "pool backward");
}

int nn_head(const __nv_bfloat16* a3, int n, const float* fw, const float* fb, float* logits, float* prob,
            const int32_t* y, float* loss, float* dfw, float* dfb, __nv_bfloat16* da3, cudaStream_t s)
{
    k_head<<<n, 64, 0, s>>>(a3, n, fw, fb, logits, prob, y, loss, dfw, dfb, da3);
    return af_cuda_check(cudaGetLastError(), "head");
}

int nn_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, int step, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<grid_for(n, 256), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return af_cuda_check(cudaGetLastError(), "adam");
}

int nn_f32_to_bf16(const float* x, int64_t n, __nv_bfloat16* y, cudaStream_t s)
{
    k_f32_to_bf16<<<grid_for(n, 256), 256, 0, s>>>(x, n, y);
    return af_cuda_check(cudaGetLastError(), "to bf16");
}
