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
// argmax (0..3, raster order) | 4 when the maximum was > 0
__global__ void k_pool_back(const __nv_bfloat16* __restrict__ dp, const uint8_t* __restrict__ idx, int n, int H,
                            int W, int c, __nv_bfloat16* __restrict__ dz)
{
    const int64_t total = (int64_t)n * H * W * c;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(e % c);
        const int64_t p = e / c;
        const int x = (int)(p % W), y = (int)((p / W) % H);
        const int64_t b = p / ((int64_t)W * H);
        const int64_t o = ((b * (H / 2) + y / 2) * (W / 2) + x / 2) * c + ch;
        float v = 0.f;
        if (idx[o] == (uint8_t)(4 | ((y & 1) * 2 + (x & 1)))) v = __bfloat162float(dp[o]);
        dz[e] = __float2bfloat16(v);
    }
}

// db[o] += sum over pixels of dz[p][o]   (dz bf16 [P][c]); block partial sums
// are reduced in shared memory, then one atomic per channel and block
__global__ void k_colsum(const __nv_bfloat16* __restrict__ dz, int64_t P, int c, float* __restrict__ db)
{
    __shared__ float part[256];
    const int ch = threadIdx.x % c;
    const int lanes = blockDim.x / c;
    float s = 0.f;
    for (int64_t p = (int64_t)blockIdx.x * lanes + threadIdx.x / c; p < P; p += (int64_t)gridDim.x * lanes)
        s += __bfloat162float(dz[p * c + ch]);
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < c) {
        float t = 0.f;
        for (int l = 0; l < lanes; l++) t += part[l * c + threadIdx.x];
        atomicAdd(db + threadIdx.x, t);
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
                 cudaStream_t s)
{
    k_pool_back<<<grid_for((int64_t)n * H * W * c, 256), 256, 0, s>>>(dp, idx, n, H, W, c, dz);
    return af_cuda_check(cudaGetLastError(), "pool backward");
}

int nn_colsum(const __nv_bfloat16* dz, int64_t P, int c, float* db, cudaStream_t s)
{
    const int threads = (256 / c) * c;
    unsigned blocks = grid_for(P, threads / c);
    if (blocks > 304) blocks = 304;
    k_colsum<<<blocks, threads, 0, s>>>(dz, P, c, db);
    return af_cuda_check(cudaGetLastError(), "bias gradient");
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
