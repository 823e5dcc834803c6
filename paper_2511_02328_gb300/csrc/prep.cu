// prep.cu -- preprocessing of the filterbank before the search (Sec. 2.2):
// square-law time downsampling and the zero-DM filter.
//
//   out[c][k] = min( sqrt(V * S / N), V ),  S = sum of bin k (N samples), V = 255,
//   rounded half up, exactly: floor((isqrt(floor(4 V S / N)) + 1) / 2), evaluated
//   as max r with r^2 N <= 4 V S from a float estimate and two integer tests.
//
// One block per (channel, run of TB bins): the block's input span is read
// with coalesced loads into shared memory, then every thread sums its bins
// there.  HBM-bound: nchan * nsamp bytes read, nchan * nsamp / D written.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace {

constexpr int kDsThreads = 256;
constexpr int kDsSpan = 32768;  // bytes of input per block (shared memory)

// The rounded square root floor((isqrt(floor(T / N)) + 1) / 2), T = 4 V S, without
// an integer division: isqrt(floor(T / N)) = max r with r^2 N <= T.  A float
// estimate (rcpN = 1/N) is within one of r; two exact integer tests settle it.
__device__ __forceinline__ uint32_t sqlaw_value(uint64_t T, uint32_t N, float rcpN)
{
    uint32_t r = (uint32_t)sqrtf((float)T * rcpN);
    if ((uint64_t)r * r * N > T) r--;
    if ((uint64_t)(r + 1) * (r + 1) * N <= T) r++;
    const uint32_t v = (r + 1) / 2;
    return v < 255u ? v : 255u;
}

// The same for D <= 16384, in 32 bits: T = 4 V S <= 4 * 255 * 255 * D < 2^32 and
// r <= 510, so r^2 N <= 260100 D < 2^32 as well.
__device__ __forceinline__ uint32_t sqlaw_value32(uint32_t T, uint32_t N, float rcpN)
{
    uint32_t r = (uint32_t)sqrtf((float)T * rcpN);
    if (r * r * N > T) r--;
    if ((r + 1) * (r + 1) * N <= T) r++;
    const uint32_t v = (r + 1) / 2;
    return v < 255u ? v : 255u;
}

__global__ void __launch_bounds__(kDsThreads)
k_downsample(const uint8_t* __restrict__ X, int64_t nsamp, int D, int64_t nout, int tb, unsigned runs,
             uint8_t* __restrict__ out)
{
    __shared__ __align__(16) uint8_t sx[kDsSpan];
    const int c = (int)(blockIdx.x / runs);
    const int64_t k0 = (int64_t)(blockIdx.x % runs) * tb;
    const int64_t t0 = k0 * D;
    const int64_t span = min((int64_t)tb * D, nsamp - t0);
    const uint8_t* x = X + (int64_t)c * nsamp + t0;
    int64_t done = 0;
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        // all of a thread's 16-byte loads are issued before the first shared store
        constexpr int NB = kDsSpan / 16 / kDsThreads;
        const int n16 = (int)(span >> 4);
        uint4 v[NB];
#pragma unroll
        for (int u = 0; u < NB; u++)
            if ((int)threadIdx.x + u * kDsThreads < n16)
                v[u] = __ldg(reinterpret_cast<const uint4*>(x) + threadIdx.x + u * kDsThreads);
#pragma unroll
        for (int u = 0; u < NB; u++)
            if ((int)threadIdx.x + u * kDsThreads < n16) reinterpret_cast<uint4*>(sx)[threadIdx.x + u * kDsThreads] = v[u];
        done = (int64_t)n16 << 4;
    }
    for (int64_t i = done + threadIdx.x; i < span; i += kDsThreads) sx[i] = __ldg(x + i);
    __syncthreads();
    const float rcpD = 1.0f / (float)D;
    const int sp = (int)span;  // <= kDsSpan: 32-bit indices from here on
    for (int k = threadIdx.x; k < tb && k0 + k < nout; k += kDsThreads) {
        const int a = k * D, b = min(a + D, sp);
        uint32_t S = 0;
        int i = a;
        if ((D & 3) == 0)  // whole 32-bit words: one dp4a per 4 samples
            for (; i + 4 <= b; i += 4) S = __dp4a(*reinterpret_cast<const uint32_t*>(sx + i), 0x01010101u, S);
        for (; i < b; i++) S += sx[i];
        const uint32_t N = (uint32_t)(b - a);
        const float rcpN = N == (uint32_t)D ? rcpD : 1.0f / (float)N;  // only the last bin is short
        out[(int64_t)c * nout + k0 + k] = D <= 16384 ? (uint8_t)sqlaw_value32(1020u * S, N, rcpN)
                                                     : (uint8_t)sqlaw_value(4ull * 255ull * S, N, rcpN);
    }
}

}  // namespace

extern "C" int af_downsample(const uint8_t* d_in, int nchan, int64_t nsamp, int D, uint8_t* d_out, void* stream)
try {
    if (!d_in || !d_out) return af_set_error(AF_EINVAL, "af_downsample: NULL buffer");
    if (nchan < 1 || nsamp < 1) return af_set_error(AF_EINVAL, "af_downsample: empty input");
    if (D < 1 || D > kDsSpan) return af_set_error(AF_EINVAL, "af_downsample: D %d not in 1..%d", D, kDsSpan);
    const int64_t nout = (nsamp + D - 1) / D;
    const int tb = kDsSpan / D;
    const int64_t runs = (nout + tb - 1) / tb;
    if ((long double)runs * nchan > 0x7fffffff) return af_set_error(AF_EINVAL, "af_downsample: input too large");
    k_downsample<<<(unsigned)(runs * nchan), kDsThreads, 0, (cudaStream_t)stream>>>(d_in, nsamp, D, nout, tb,
                                                                                    (unsigned)runs, d_out);
    return af_cuda_check(cudaGetLastError(), "af_downsample launch");
} catch (...) {
    return af_host_exception("af_downsample");
}

// ---------------------------------------------------------------- zero-DM
// Zero-DM filter: q[t] = round_half_up(sum_c X[c][t] / nchan), out = clip(X - q + 128).
// Fast path (rows 16-byte aligned, nsamp % 16 == 0): a block owns a tile of
// 512 samples; its 16 warps split the channels, lane l holding samples
// [16 l, 16 l + 16) of the tile as one 16-byte load per channel.
//   pass 1: per-warp channel sums in 16-bit lanes (bytes 0,2 / 1,3 of each
//           word, folded into 32-bit sums every 256 channels), reduced across
//           warps in shared memory into q[512];
//   pass 2: every warp re-reads its channels and writes clip(x - q + 128).
// In place is safe: a block reads every channel of its tile before writing.
// Other shapes: one thread per 4 samples of every channel, byte accesses.
namespace {

constexpr int kZW = 16;           // warps per block (channel split)
constexpr int kZTile = 512;       // samples per block
constexpr int kZT = 128;          // generic kernel: threads per block

__global__ void __launch_bounds__(kZW * 32)
k_zerodm16(const uint8_t* X, int nchan, int64_t nsamp, uint8_t* out)
{
    __shared__ uint32_t part[kZW][kZTile];
    __shared__ int32_t q[kZTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t0 = (int64_t)blockIdx.x * kZTile + 16 * lane;
    const int c0 = (int)((int64_t)nchan * warp / kZW), c1 = (int)((int64_t)nchan * (warp + 1) / kZW);
    uint32_t sum[16];
#pragma unroll
    for (int i = 0; i < 16; i++) sum[i] = 0u;
    for (int cb = c0; cb < c1; cb += 256) {
        const int ce = min(c1, cb + 256);
        uint32_t E[4] = {0u, 0u, 0u, 0u}, O[4] = {0u, 0u, 0u, 0u};
#pragma unroll 4
        for (int c = cb; c < ce; c++) {
            const uint4 v = *reinterpret_cast<const uint4*>(X + (int64_t)c * nsamp + t0);
            const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                E[j] += wv[j] & 0x00FF00FFu;
                O[j] += __byte_perm(wv[j], 0u, 0x4341);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            sum[4 * j + 0] += E[j] & 0xFFFFu;
            sum[4 * j + 1] += O[j] & 0xFFFFu;
            sum[4 * j + 2] += E[j] >> 16;
            sum[4 * j + 3] += O[j] >> 16;
        }
    }
#pragma unroll
    for (int i = 0; i < 16; i++) part[warp][16 * lane + i] = sum[i];
    __syncthreads();
    for (int i = threadIdx.x; i < kZTile; i += kZW * 32) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kZW; w++) s += part[w][i];
        q[i] = (int32_t)((2u * s + (uint32_t)nchan) / (2u * (uint32_t)nchan)) - 128;
    }
    __syncthreads();
    int32_t qq[16];
#pragma unroll
    for (int i = 0; i < 16; i++) qq[i] = q[16 * lane + i];
#pragma unroll 4
    for (int c = c0; c < c1; c++) {
        const int64_t o = (int64_t)c * nsamp + t0;
        const uint4 v = *reinterpret_cast<const uint4*>(X + o);  // plain load: X may alias out
        const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
        uint32_t r[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            uint32_t acc = 0;
#pragma unroll
            for (int b = 0; b < 4; b++) {
                const int x = (int)((wv[j] >> (8 * b)) & 0xFFu) - qq[4 * j + b];
                acc |= (uint32_t)min(255, max(0, x)) << (8 * b);
            }
            r[j] = acc;
        }
        *reinterpret_cast<uint4*>(out + o) = make_uint4(r[0], r[1], r[2], r[3]);
    }
}

__global__ void __launch_bounds__(kZT)
k_zerodm(const uint8_t* X, int nchan, int64_t nsamp, uint8_t* out)
{
    const int64_t t = ((int64_t)blockIdx.x * kZT + threadIdx.x) * 4;
    if (t >= nsamp) return;
    const int n = (int)min((int64_t)4, nsamp - t);
    uint32_t s[4] = {0u, 0u, 0u, 0u};
    for (int c = 0; c < nchan; c++)
        for (int i = 0; i < n; i++) s[i] += X[(int64_t)c * nsamp + t + i];
    int q[4];
#pragma unroll
    for (int i = 0; i < 4; i++) q[i] = (int)((2u * s[i] + (uint32_t)nchan) / (2u * (uint32_t)nchan)) - 128;
    for (int c = 0; c < nchan; c++)
        for (int i = 0; i < n; i++) {
            const int64_t o = (int64_t)c * nsamp + t + i;
            const int v = (int)X[o] - q[i];
            out[o] = (uint8_t)min(255, max(0, v));
        }
}

}  // namespace

extern "C" int af_zerodm(const uint8_t* d_in, int nchan, int64_t nsamp, uint8_t* d_out, void* stream)
try {
    if (!d_in || !d_out) return af_set_error(AF_EINVAL, "af_zerodm: NULL buffer");
    if (nchan < 1 || nchan > 65536 || nsamp < 1) return af_set_error(AF_EINVAL, "af_zerodm: bad shape");
    cudaStream_t s = (cudaStream_t)stream;
    const bool fast = nsamp % kZTile == 0 && ((uintptr_t)d_in % 16 == 0) && ((uintptr_t)d_out % 16 == 0) &&
                      nchan >= kZW;
    if (fast) {
        const int64_t blocks = nsamp / kZTile;
        if (blocks > 0x7fffffff) return af_set_error(AF_EINVAL, "af_zerodm: input too large");
        k_zerodm16<<<(unsigned)blocks, kZW * 32, 0, s>>>(d_in, nchan, nsamp, d_out);
    } else {
        const int64_t blocks = (nsamp + 4 * kZT - 1) / (4 * kZT);
        if (blocks > 0x7fffffff) return af_set_error(AF_EINVAL, "af_zerodm: input too large");
        k_zerodm<<<(unsigned)blocks, kZT, 0, s>>>(d_in, nchan, nsamp, d_out);
    }
    return af_cuda_check(cudaGetLastError(), "af_zerodm launch");
} catch (...) {
    return af_host_exception("af_zerodm");
}
