// prep.cu -- preprocessing of the filterbank before the search (Sec. 2.2):
// square-law time downsampling and the zero-DM filter.
//
//   out[c][k] = min( sqrt(V * S / N), V ),  S = sum of bin k (N samples), V = 255,
//   rounded half up, exactly: floor((isqrt(floor(4 V S / N)) + 1) / 2).
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

// isqrt(q) for q < 2^24: the float square root (correctly rounded) is within
// one of the integer root; the two integer tests settle it exactly.
__device__ __forceinline__ uint32_t isqrt_small(uint32_t q)
{
    uint32_t r = (uint32_t)sqrtf((float)q);
    if (r * r > q) r--;
    if ((r + 1) * (r + 1) <= q) r++;
    return r;
}

__global__ void __launch_bounds__(kDsThreads)
k_downsample(const uint8_t* __restrict__ X, int64_t nsamp, int D, int64_t nout, int tb, unsigned runs,
             uint8_t* __restrict__ out)
{
    __shared__ uint8_t sx[kDsSpan];
    const int c = (int)(blockIdx.x / runs);
    const int64_t k0 = (int64_t)(blockIdx.x % runs) * tb;
    const int64_t t0 = k0 * D;
    const int64_t span = min((int64_t)tb * D, nsamp - t0);
    const uint8_t* x = X + (int64_t)c * nsamp + t0;
    for (int64_t i = threadIdx.x; i < span; i += kDsThreads) sx[i] = __ldg(x + i);
    __syncthreads();
    for (int k = threadIdx.x; k < tb && k0 + k < nout; k += kDsThreads) {
        const int64_t a = (int64_t)k * D, b = min(a + D, span);
        uint32_t S = 0;
        for (int64_t i = a; i < b; i++) S += sx[i];
        const uint32_t N = (uint32_t)(b - a);
        const uint32_t q = (uint32_t)((4ull * 255ull * S) / N);  // <= 4 * 255 * 255
        const uint32_t v = (isqrt_small(q) + 1) / 2;
        out[(int64_t)c * nout + k0 + k] = (uint8_t)min(v, 255u);
    }
}

}  // namespace

extern "C" int af_downsample(const uint8_t* d_in, int nchan, int64_t nsamp, int D, uint8_t* d_out, void* stream)
{
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
}

// ---------------------------------------------------------------- zero-DM
// Zero-DM filter: q[t] = round_half_up(sum_c X[c][t] / nchan), out = clip(X - q + 128).
// Each thread owns 4 consecutive samples of every channel: it sums the column
// block over all channels, then rewrites it (in place is safe: no thread reads
// another thread's samples).  Word loads when the rows are 4-byte aligned.
namespace {

constexpr int kZT = 128;

__global__ void __launch_bounds__(kZT)
k_zerodm(const uint8_t* X, int nchan, int64_t nsamp, uint8_t* out, int aligned)
{
    const int64_t t = ((int64_t)blockIdx.x * kZT + threadIdx.x) * 4;
    if (t >= nsamp) return;
    const int n = (int)min((int64_t)4, nsamp - t);
    uint32_t s[4] = {0u, 0u, 0u, 0u};
    if (aligned && n == 4) {
#pragma unroll 8
        for (int c = 0; c < nchan; c++) {
            const uint32_t w = *reinterpret_cast<const uint32_t*>(X + (int64_t)c * nsamp + t);
            s[0] += w & 0xFFu;
            s[1] += (w >> 8) & 0xFFu;
            s[2] += (w >> 16) & 0xFFu;
            s[3] += w >> 24;
        }
    } else {
        for (int c = 0; c < nchan; c++)
            for (int i = 0; i < n; i++) s[i] += X[(int64_t)c * nsamp + t + i];
    }
    int q[4];
#pragma unroll
    for (int i = 0; i < 4; i++) q[i] = (int)((2u * s[i] + (uint32_t)nchan) / (2u * (uint32_t)nchan)) - 128;
    if (aligned && n == 4) {
#pragma unroll 8
        for (int c = 0; c < nchan; c++) {
            const int64_t o = (int64_t)c * nsamp + t;
            const uint32_t w = *reinterpret_cast<const uint32_t*>(X + o);
            uint32_t r = 0;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int v = (int)((w >> (8 * i)) & 0xFFu) - q[i];
                r |= (uint32_t)min(255, max(0, v)) << (8 * i);
            }
            *reinterpret_cast<uint32_t*>(out + o) = r;
        }
    } else {
        for (int c = 0; c < nchan; c++)
            for (int i = 0; i < n; i++) {
                const int64_t o = (int64_t)c * nsamp + t + i;
                const int v = (int)X[o] - q[i];
                out[o] = (uint8_t)min(255, max(0, v));
            }
    }
}

}  // namespace

extern "C" int af_zerodm(const uint8_t* d_in, int nchan, int64_t nsamp, uint8_t* d_out, void* stream)
{
    if (!d_in || !d_out) return af_set_error(AF_EINVAL, "af_zerodm: NULL buffer");
    if (nchan < 1 || nchan > 65536 || nsamp < 1) return af_set_error(AF_EINVAL, "af_zerodm: bad shape");
    const int64_t blocks = (nsamp + 4 * kZT - 1) / (4 * kZT);
    if (blocks > 0x7fffffff) return af_set_error(AF_EINVAL, "af_zerodm: input too large");
    const int aligned = (nsamp % 4 == 0) && ((uintptr_t)d_in % 4 == 0) && ((uintptr_t)d_out % 4 == 0);
    k_zerodm<<<(unsigned)blocks, kZT, 0, (cudaStream_t)stream>>>(d_in, nchan, nsamp, d_out, aligned);
    return af_cuda_check(cudaGetLastError(), "af_zerodm launch");
}
