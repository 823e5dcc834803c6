// nn.cu -- kernels of the candidate classifier (replaces the paper's YOLO
// detector, Sec. 2.5): a BF16 tensor-core GEMM with FP32 accumulation that
// serves the forward, data-gradient and weight-gradient passes of 3x3
// convolutions, plus im2col / col2im, 2x2 max pooling, the classifier head,
// and Adam.
//
// GEMM: C[M][N] = sum_k A[m][k] B[k][n], operands in shared memory, fed to
// mma.sync.m16n8k16 (bf16 x bf16 -> f32) with ldmatrix.  Each operand is
// either K-contiguous (A[m][k] / B^T[n][k]) or M/N-contiguous (A^T[k][m] /
// B[k][n]); the latter are loaded with ldmatrix.trans, so
//   forward   Z  = col  x W^T      A = col [NHW][Kp] (K-major), B = W [Cout][Kp] (K-major)
//   dgrad     dcol = dZ x W       A = dZ [NHW][Cout] (K-major), B = W [Cout][Kp] (N-major)
//   wgrad     dW = dZ^T x col     A = dZ [NHW][Cout] (M-major), B = col [NHW][Kp] (N-major)
// need no transposed copies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "nn.h"

namespace {

constexpr int BM = 64, BN = 64, BK = 32, GT = 128;  // 4 warps, 2 x 2, 32 x 32 each
constexpr int PADK = 8, PADM = 8;

template <bool AK, bool BK_>
struct Smem {
    // A: K-major -> [BM][BK+PADK]; M-major -> [BK][BM+PADM].  Same for B with N.
    static constexpr int A_ELEMS = AK ? BM * (BK + PADK) : BK * (BM + PADM);
    static constexpr int B_ELEMS = BK_ ? BN * (BK + PADK) : BK * (BN + PADM);
};

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Loads one BK slice of an operand tile into shared memory.  `ld` is the row
// pitch in elements (multiple of 8); out-of-range rows / k are zero.
//   KMAJ: rows = the M (or N) index, BK contiguous k per row
//   else: rows = k, BM contiguous m per row
template <bool KMAJ, int R>
__device__ __forceinline__ void load_tile(__nv_bfloat16* s, const __nv_bfloat16* g, int ld, int r0, int rlim, int k0,
                                          int klim)
{
    if (KMAJ) {
        // R rows x BK cols, 16-byte chunks: R * BK / 8 chunks
        for (int c = threadIdx.x; c < R * BK / 8; c += GT) {
            const int r = c / (BK / 8), kc = (c % (BK / 8)) * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (r0 + r < rlim && k0 + kc < klim)
                v = *reinterpret_cast<const uint4*>(g + (int64_t)(r0 + r) * ld + k0 + kc);
            *reinterpret_cast<uint4*>(s + r * (BK + PADK) + kc) = v;
        }
    } else {
        // BK rows (k) x R cols
        for (int c = threadIdx.x; c < BK * R / 8; c += GT) {
            const int k = c / (R / 8), rc = (c % (R / 8)) * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (k0 + k < klim && r0 + rc < rlim)
                v = *reinterpret_cast<const uint4*>(g + (int64_t)(k0 + k) * ld + r0 + rc);
            *reinterpret_cast<uint4*>(s + k * (R + PADM) + rc) = v;
        }
    }
}

template <bool AK, bool BKM, int EPI>
__global__ void __launch_bounds__(GT) k_gemm(const __nv_bfloat16* __restrict__ A, int lda,
                                             const __nv_bfloat16* __restrict__ B, int ldb, int M, int N, int K,
                                             int kchunk, float* __restrict__ C, int ldc,
                                             const float* __restrict__ bias)
{
    __shared__ __align__(16) __nv_bfloat16 sA[Smem<AK, BKM>::A_ELEMS];
    __shared__ __align__(16) __nv_bfloat16 sB[Smem<AK, BKM>::B_ELEMS];
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[i][j][q] = 0.f;
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(sA), sb = (uint32_t)__cvta_generic_to_shared(sB);

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        load_tile<AK, BM>(sA, A, lda, m0, M, k0, kend);
        load_tile<BKM, BN>(sB, B, ldb, n0, N, k0, kend);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int mb = wm + 16 * i;
                if (AK) {
                    const int row = mb + (lane & 15), col = kk + (lane >> 4) * 8;
                    ldsm_x4(sa + 2 * (row * (BK + PADK) + col), a[i][0], a[i][1], a[i][2], a[i][3]);
                } else {
                    const int krow = kk + (lane & 7) + ((lane >> 4) & 1) * 8, col = mb + ((lane >> 3) & 1) * 8;
                    ldsm_x4_t(sa + 2 * (krow * (BM + PADM) + col), a[i][0], a[i][1], a[i][2], a[i][3]);
                }
            }
#pragma unroll
            for (int jj = 0; jj < 2; jj++) {
                const int nb = wn + 16 * jj;
                uint32_t r0, r1, r2, r3;
                if (BKM) {
                    const int row = nb + (lane & 7) + ((lane >> 4) & 1) * 8, col = kk + ((lane >> 3) & 1) * 8;
                    ldsm_x4(sb + 2 * (row * (BK + PADK) + col), r0, r1, r2, r3);
                } else {
                    const int krow = kk + (lane & 7) + ((lane >> 3) & 1) * 8, col = nb + ((lane >> 4) & 1) * 8;
                    ldsm_x4_t(sb + 2 * (krow * (BN + PADM) + col), r0, r1, r2, r3);
                }
                b[2 * jj][0] = r0;
                b[2 * jj][1] = r1;
                b[2 * jj + 1][0] = r2;
                b[2 * jj + 1][1] = r3;
            }
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) mma_bf16(acc[i][j], a[i], b[j][0], b[j][1]);
        }
        __syncthreads();
    }
    const int g = lane >> 2, tg = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int m = m0 + wm + 16 * i + g + 8 * h;
                const int n = n0 + wn + 8 * j + 2 * tg;
                if (m >= M) continue;
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    if (n + e >= N) continue;
                    float v = acc[i][j][2 * h + e];
                    float* dst = C + (int64_t)m * ldc + n + e;
                    if (EPI == NN_EPI_STORE) {
                        *dst = v;
                    } else if (EPI == NN_EPI_BIAS_RELU) {
                        v += bias[n + e];
                        *dst = v > 0.f ? v : 0.f;
                    } else {
                        atomicAdd(dst, v);
                    }
                }
            }
}

// --------------------------------------------------------------- conv helpers
// col[p][k] for pixel p = (n, y, x), k = (dy * 3 + dx) * cin + i  (k >= 9 cin: 0)
__global__ void k_im2col(const __nv_bfloat16* __restrict__ a, int n, int H, int W, int cin, int kp,
                         __nv_bfloat16* __restrict__ col)
{
    const int64_t total = (int64_t)n * H * W * kp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % kp);
        const int64_t p = e / kp;
        const int x = (int)(p % W), y = (int)((p / W) % H);
        const int64_t b = p / ((int64_t)W * H);
        __nv_bfloat16 v = __float2bfloat16(0.f);
        if (k < 9 * cin) {
            const int tap = k / cin, i = k % cin;
            const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) v = a[((b * H + yy) * W + xx) * cin + i];
        }
        col[e] = v;
    }
}

// da[n][y][x][i] = sum_{dy,dx} dcol[(n, y-dy+1, x-dx+1)][(dy*3+dx)*cin + i], rounded to bf16
__global__ void k_col2im(const float* __restrict__ dcol, int n, int H, int W, int cin, int kp,
                         __nv_bfloat16* __restrict__ da)
{
    const int64_t total = (int64_t)n * H * W * cin;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % cin);
        const int64_t p = e / cin;
        const int x = (int)(p % W), y = (int)((p / W) % H);
        const int64_t b = p / ((int64_t)W * H);
        float s = 0.f;
        for (int tap = 0; tap < 9; tap++) {
            const int yy = y - (tap / 3 - 1), xx = x - (tap % 3 - 1);
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) s += dcol[((b * H + yy) * W + xx) * kp + tap * cin + i];
        }
        da[e] = __float2bfloat16(s);
    }
}

// 2x2 max pool of r [n][H][W][c] (fp32) -> out bf16 [n][H/2][W/2][c] and the
// argmax (0..3 in raster order, first maximum wins)
__global__ void k_pool(const float* __restrict__ r, int n, int H, int W, int c, __nv_bfloat16* __restrict__ out,
                       uint8_t* __restrict__ idx)
{
    const int Ho = H / 2, Wo = W / 2;
    const int64_t total = (int64_t)n * Ho * Wo * c;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(e % c);
        const int64_t p = e / c;
        const int xo = (int)(p % Wo), yo = (int)((p / Wo) % Ho);
        const int64_t b = p / ((int64_t)Wo * Ho);
        float best = -INFINITY;
        int bi = 0;
        for (int q = 0; q < 4; q++) {
            const float v = r[((b * H + 2 * yo + q / 2) * W + 2 * xo + q % 2) * c + ch];
            if (v > best) {
                best = v;
                bi = q;
            }
        }
        out[e] = __float2bfloat16(best);
        idx[e] = (uint8_t)bi;
    }
}

// dz [n][H][W][c] (bf16) = (pooled gradient routed to the argmax) * (r > 0)
__global__ void k_pool_back(const __nv_bfloat16* __restrict__ dp, const uint8_t* __restrict__ idx,
                            const float* __restrict__ r, int n, int H, int W, int c, __nv_bfloat16* __restrict__ dz)
{
    const int64_t total = (int64_t)n * H * W * c;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(e % c);
        const int64_t p = e / c;
        const int x = (int)(p % W), y = (int)((p / W) % H);
        const int64_t b = p / ((int64_t)W * H);
        const int64_t o = ((b * (H / 2) + y / 2) * (W / 2) + x / 2) * c + ch;
        float v = 0.f;
        if (idx[o] == (uint8_t)((y & 1) * 2 + (x & 1)) && r[e] > 0.f) v = __bfloat162float(dp[o]);
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

// dW [cout][kp] fp32 -> grad [cout][9 cin]
__global__ void k_unpack_dw(const float* __restrict__ dw, int cout, int k9, int kp, float* __restrict__ g)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cout * k9) return;
    g[e] = dw[(e / k9) * kp + e % k9];
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

template <bool AK, bool BKM, int EPI>
static int launch_gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                       int splits, float* C, int ldc, const float* bias, cudaStream_t s)
{
    int kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + BK - 1) / BK * BK;
    splits = (K + kchunk - 1) / kchunk;
    dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN, splits);
    k_gemm<AK, BKM, EPI><<<grid, GT, 0, s>>>(A, lda, B, ldb, M, N, K, kchunk, C, ldc, bias);
    return af_cuda_check(cudaGetLastError(), "gemm launch");
}

int nn_gemm(int layout, int epi, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
            int splits, float* C, int ldc, const float* bias, cudaStream_t s)
{
    if ((lda & 7) || (ldb & 7) || (K & 7) || ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || M < 1 || N < 1 || K < 1 ||
        splits < 1)
        return af_set_error(AF_EINVAL,
                            "gemm: K and the leading dimensions must be multiples of 8, operands 16-byte aligned");
    if (epi != NN_EPI_ATOMIC) splits = 1;
#define AF_GEMM_CASE(L, AKv, BKv)                                                                               \
    case L:                                                                                                     \
        if (epi == NN_EPI_STORE) return launch_gemm<AKv, BKv, NN_EPI_STORE>(A, lda, B, ldb, M, N, K, 1, C, ldc, bias, s); \
        if (epi == NN_EPI_BIAS_RELU)                                                                            \
            return launch_gemm<AKv, BKv, NN_EPI_BIAS_RELU>(A, lda, B, ldb, M, N, K, 1, C, ldc, bias, s);        \
        return launch_gemm<AKv, BKv, NN_EPI_ATOMIC>(A, lda, B, ldb, M, N, K, splits, C, ldc, bias, s);
    switch (layout) {
        AF_GEMM_CASE(NN_A_K_B_K, true, true)
        AF_GEMM_CASE(NN_A_K_B_N, true, false)
        AF_GEMM_CASE(NN_A_M_B_N, false, false)
        AF_GEMM_CASE(NN_A_M_B_K, false, true)
    }
#undef AF_GEMM_CASE
    return af_set_error(AF_EINVAL, "gemm: unknown layout");
}

int nn_im2col(const __nv_bfloat16* a, int n, int H, int W, int cin, int kp, __nv_bfloat16* col, cudaStream_t s)
{
    k_im2col<<<grid_for((int64_t)n * H * W * kp, 256), 256, 0, s>>>(a, n, H, W, cin, kp, col);
    return af_cuda_check(cudaGetLastError(), "im2col");
}

int nn_col2im(const float* dcol, int n, int H, int W, int cin, int kp, __nv_bfloat16* da, cudaStream_t s)
{
    k_col2im<<<grid_for((int64_t)n * H * W * cin, 256), 256, 0, s>>>(dcol, n, H, W, cin, kp, da);
    return af_cuda_check(cudaGetLastError(), "col2im");
}

int nn_pool(const float* r, int n, int H, int W, int c, __nv_bfloat16* out, uint8_t* idx, cudaStream_t s)
{
    k_pool<<<grid_for((int64_t)n * H * W * c / 4, 256), 256, 0, s>>>(r, n, H, W, c, out, idx);
    return af_cuda_check(cudaGetLastError(), "pool");
}

int nn_pool_back(const __nv_bfloat16* dp, const uint8_t* idx, const float* r, int n, int H, int W, int c,
                 __nv_bfloat16* dz, cudaStream_t s)
{
    k_pool_back<<<grid_for((int64_t)n * H * W * c, 256), 256, 0, s>>>(dp, idx, r, n, H, W, c, dz);
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

int nn_unpack_dw(const float* dw, int cout, int k9, int kp, float* g, cudaStream_t s)
{
    k_unpack_dw<<<(cout * k9 + 255) / 256, 256, 0, s>>>(dw, cout, k9, kp, g);
    return af_cuda_check(cudaGetLastError(), "unpack weight gradient");
}

int nn_f32_to_bf16(const float* x, int64_t n, __nv_bfloat16* y, cudaStream_t s)
{
    k_f32_to_bf16<<<grid_for(n, 256), 256, 0, s>>>(x, n, y);
    return af_cuda_check(cudaGetLastError(), "to bf16");
}
