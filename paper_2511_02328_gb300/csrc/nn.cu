// nn.cu -- elementwise and reduction kernels of the candidate classifier
// (replaces the paper's YOLO detector, Sec. 2.5): the 2x2 max-pool backward
// pass, the bias gradient, the classifier head (global average pool, fully
// connected layer, softmax cross-entropy), Adam, and the weight packing for
// the tensor-core convolutions of conv_umma.cu.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "nn.h"

namespace {

// dz [n][H][W][c] (bf16) = the pooled gradient routed to the argmax of each
// 2x2 window where that maximum (a ReLU output) was positive: idx holds the
// argmax (0..3, raster order) | 4 when the maximum was > 0.  Thread = (pooled
// pixel, 8 channels): one 16-byte load of the pooled gradient, one 8-byte load
// of the argmax bytes, four 16-byte stores.  The bias gradient (the sum of dz
// over all pixels, i.e. of the routed values) is accumulated on the way:
// per-thread sums, reduced per block in shared memory, one atomic per channel
// and block.
__global__ void __launch_bounds__(256) k_pool_back(const __nv_bfloat16* __restrict__ dp, const uint8_t* __restrict__ idx,
                                                   int n, int H, int W, int c, __nv_bfloat16* __restrict__ dz,
                                                   float* __restrict__ db)
{
    __shared__ float part[256][8];
    const int Ho = H / 2, Wo = W / 2, cg = c / 8;
    const int64_t total = (int64_t)n * Ho * Wo * cg;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;  // a multiple of cg: each thread keeps its group
    const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) % cg);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int64_t pp = e / cg;
        const int xo = (int)(pp % Wo);
        const int64_t r = pp / Wo;  // img * Ho + yo
        const uint4 v = *reinterpret_cast<const uint4*>(dp + pp * c + 8 * g);
        const uint2 ix = *reinterpret_cast<const uint2*>(idx + pp * c + 8 * g);
        const uint16_t* vv = reinterpret_cast<const uint16_t*>(&v);
        const uint8_t* ii = reinterpret_cast<const uint8_t*>(&ix);
#pragma unroll
        for (int j = 0; j < 8; j++)
            if (ii[j] & 4) acc[j] += __bfloat162float(__ushort_as_bfloat16(vv[j]));
#pragma unroll
        for (int q = 0; q < 4; q++) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t lo = ii[2 * j] == (uint8_t)(4 | q) ? vv[2 * j] : 0u;
                const uint32_t hi = ii[2 * j + 1] == (uint8_t)(4 | q) ? vv[2 * j + 1] : 0u;
                w[j] = lo | (hi << 16);
            }
            const int64_t p = (2 * r + (q >> 1)) * W + 2 * xo + (q & 1);  // (img * H + y) * W + x
            *reinterpret_cast<uint4*>(dz + p * c + 8 * g) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
#pragma unroll
    for (int j = 0; j < 8; j++) part[threadIdx.x][j] = acc[j];
    __syncthreads();
    if ((int)threadIdx.x < c) {
        // channel ch = 8 gg + j is summed by the threads t with t % cg == gg
        const int gg = threadIdx.x / 8, j = threadIdx.x % 8;
        float sum = 0.f;
        for (int t = gg; t < (int)blockDim.x; t += cg) sum += part[t][j];  // 256 % cg == 0: thread t has group t % cg
        atomicAdd(db + threadIdx.x, sum);
    }
}

// Head: per sample, global average pool of a3 [n][64 positions][64] (bf16),
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
    const __nv_bfloat16* a = a3 + (int64_t)s * 64 * 64;
    float acc = 0.f;
    for (int q = 0; q < 64; q++) acc += __bfloat162float(a[q * 64 + ch]);
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
    for (int q = 0; q < 64; q++) da3[(int64_t)s * 4096 + q * 64 + ch] = v;
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

// fp32 master weights [cout][9*cin] -> bf16 [cout][kp] (zero padding)
__global__ void k_pack_w(const float* __restrict__ w, int cout, int k9, int kp, __nv_bfloat16* __restrict__ wt)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cout * kp) return;
    const int o = e / kp, k = e % kp;
    wt[e] = __float2bfloat16(k < k9 ? w[o * k9 + k] : 0.f);
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
    if (c % 8 || c > 256 || ((uintptr_t)dp & 15) || ((uintptr_t)dz & 15) || ((uintptr_t)idx & 7))
        return af_set_error(AF_EINVAL, "pool backward: channels / alignment");
    const int64_t total = (int64_t)n * (H / 2) * (W / 2) * (c / 8);
    k_pool_back<<<grid_for(total, 256), 256, 0, s>>>(dp, idx, n, H, W, c, dz, db);
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

int nn_pack_w(const float* w, int cout, int k9, int kp, __nv_bfloat16* wt, cudaStream_t s)
{
    k_pack_w<<<(cout * kp + 255) / 256, 256, 0, s>>>(w, cout, k9, kp, wt);
    return af_cuda_check(cudaGetLastError(), "pack weights");
}

int nn_f32_to_bf16(const float* x, int64_t n, __nv_bfloat16* y, cudaStream_t s)
{
    k_f32_to_bf16<<<grid_for(n, 256), 256, 0, s>>>(x, n, y);
    return af_cuda_check(cudaGetLastError(), "to bf16");
}
