// snr.cu -- boxcar matched filter and S/N normalisation (step (iii) of the
// single-pulse workflow, Sec. 1 of the paper; definitions as in afgb.h).
//
//   B_w[t]  = sum_{k=t}^{t+w-1} Y[d][k]
//   snr_w   = (nout*B_w - w*S) / (nout*sigma*sqrt(w))
//           = (B_w - q_w) * k_w - c_w,   q_w = floor(w*S/nout),
//             k_w = 1/(sigma*sqrt(w)),  c_w = ((w*S - q_w*nout)/nout) * k_w
//
// The split keeps the cancellation B_w - w*mu exact in integers: (B_w - q_w)
// is an exact integer and only the final scale is rounded, so the float
// result is within a few ulp of the exact S/N.  Window sums come from 32-bit
// prefix sums taken modulo 2^32, which are exact as long as every window sum
// is below 2^32 (checked on the host: w * 255 * nchan < 2^32).
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace {

__device__ __forceinline__ double i128_to_double(__int128 v)
{
    const bool neg = v < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const double r = (double)(uint64_t)(u >> 64) * 18446744073709551616.0 + (double)(uint64_t)u;
    return neg ? -r : r;
}

// One thread per (row, width): the constants q, k, c above, from the exact
// row sums.  sigma^2 = (nout*Q - S^2)/nout^2 with the numerator in 128 bits.
__global__ void k_rowconst(const af_rowstats_t* __restrict__ st, int ndm, int64_t nout, af_widths_t w,
                           af_rowconst_t* __restrict__ rc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ndm * w.n) return;
    const int d = i / w.n, wi = i % w.n;
    const int64_t S = st[d].sum, Q = st[d].sumsq;
    const __int128 vnum = (__int128)nout * Q - (__int128)S * S;
    const double var = i128_to_double(vnum) / ((double)nout * (double)nout);
    const double sigma = var > 0.0 ? sqrt(var) : 0.0;
    const int64_t W = w.w[wi];
    const int64_t ws = W * S;            // < nout * 2^32 <= 2^63 by the width check
    const int64_t q = ws / nout;         // S >= 0: truncation is the floor
    const int64_t r = ws - q * nout;     // 0 <= r < nout
    af_rowconst_t o;
    o.q = q;
    if (sigma > 0.0) {
        const double k = 1.0 / (sigma * sqrt((double)W));
        o.k = (float)k;
        o.c = (float)(((double)r / (double)nout) * k);
    } else {
        o.k = 0.0f;
        o.c = 0.0f;
    }
    rc[(int64_t)d * AF_MAX_WIDTHS + wi] = o;
}

constexpr int kBT = 256;             // threads per block
constexpr int kBOut = 2048;          // outputs per block (8 per thread)
constexpr int kPer = kBOut / kBT;

// Block = one tile of one row.  Loads Y[t0 .. t0+kBOut+wmax-1) into shared
// memory, scans it into 32-bit prefix sums P[j] = sum_{k<j} Y[t0+k] (mod 2^32),
// then every output evaluates all widths from two prefix values each.
__global__ void __launch_bounds__(kBT)
k_boxcar(const int32_t* __restrict__ Y, int64_t nout, unsigned tiles, af_widths_t w,
         const af_rowconst_t* __restrict__ rc, float* __restrict__ snr, uint8_t* __restrict__ bw)
{
    extern __shared__ uint32_t sP[];
    __shared__ int64_t sq[AF_MAX_WIDTHS];
    __shared__ float sk[AF_MAX_WIDTHS], sc[AF_MAX_WIDTHS];
    __shared__ uint32_t swarp[kBT / 32];

    const int d = (int)(blockIdx.x / tiles);
    const int64_t t0 = (int64_t)(blockIdx.x % tiles) * kBOut;
    const int nw = w.n;
    const int wmax = w.w[nw - 1];
    const int64_t lend = min(nout, t0 + kBOut + wmax - 1);
    const int L = (int)(lend - t0);
    const int32_t* y = Y + (int64_t)d * nout + t0;

    if (threadIdx.x < nw) {
        const af_rowconst_t c = rc[(int64_t)d * AF_MAX_WIDTHS + threadIdx.x];
        sq[threadIdx.x] = c.q;
        sk[threadIdx.x] = c.k;
        sc[threadIdx.x] = c.c;
    }
    if (threadIdx.x == 0) sP[0] = 0u;

    // inclusive scan in chunks of kBT elements: sP[j+1] = sum_{k<=j} y[k]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (int base = 0; base < L; base += kBT) {
        const int j = base + threadIdx.x;
        uint32_t v = j < L ? (uint32_t)__ldg(y + j) : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += n;
        }
        if (lane == 31) swarp[warp] = v;
        __syncthreads();
        uint32_t off = carry;
        for (int k = 0; k < warp; k++) off += swarp[k];
        if (j < L) sP[j + 1] = v + off;
        uint32_t tot = 0;
#pragma unroll
        for (int k = 0; k < kBT / 32; k++) tot += swarp[k];
        carry += tot;
        __syncthreads();
    }

#pragma unroll 1
    for (int i = 0; i < kPer; i++) {
        const int lt = i * kBT + threadIdx.x;
        const int64_t t = t0 + lt;
        if (t >= nout) break;
        const uint32_t p0 = sP[lt];
        float best = -INFINITY;
        int bi = AF_NO_WIDTH;
        for (int k = 0; k < nw; k++) {
            const int ww = w.w[k];
            if (t + ww > nout) break;
            const uint32_t B = sP[lt + ww] - p0;
            const float v = fmaf((float)((int64_t)B - sq[k]), sk[k], -sc[k]);
            if (v > best) {
                best = v;
                bi = k;
            }
        }
        const int64_t o = (int64_t)d * nout + t;
        snr[o] = best;
        if (bw) bw[o] = (uint8_t)bi;
    }
}

// ---------------------------------------------------------------- robust S/N
// Per-row median and MAD (lower medians, exact) by radix selection: one block
// per row; each pass histograms the remaining value range into at most 2048
// bins in shared memory and keeps the bin holding the wanted rank, so a range
// of R values takes ceil(log2(R) / 11) passes (two for 20-bit rows).
constexpr int kRT = 512;
constexpr int kRB = 2048;

template <int MODE>  // 0: u = v - base;  1: u = |v - base|
__device__ __forceinline__ uint32_t robust_key(int32_t v, int32_t base)
{
    if (MODE == 0) return (uint32_t)(v - base);
    return v >= base ? (uint32_t)(v - base) : (uint32_t)(base - v);
}

// rank-th smallest key among the row's values (0-based), keys in [0, range].
template <int MODE>
__device__ uint32_t robust_select(const int32_t* __restrict__ y, int64_t n, int32_t base, uint32_t range,
                                  int64_t rank, uint32_t* hist, long long* sel)
{
    uint32_t start = 0;
    uint64_t width = (uint64_t)range + 1;
    const int tid = threadIdx.x, lane = tid & 31;
    while (width > 1) {
        const int bits = 64 - __clzll((long long)(width - 1));
        const int s = bits > 11 ? bits - 11 : 0;
        for (int i = tid; i < kRB; i += kRT) hist[i] = 0u;
        __syncthreads();
        for (int64_t t = tid; t < n; t += kRT) {
            const uint32_t u = robust_key<MODE>(__ldg(y + t), base);
            if (u >= start && (uint64_t)(u - start) < width) atomicAdd(&hist[(u - start) >> s], 1u);
        }
        __syncthreads();
        if (tid < 32) {
            // lane l owns bins [64 l, 64 l + 64): find the bin where the count passes rank
            uint32_t own = 0;
            for (int i = 0; i < 64; i++) own += hist[lane * 64 + i];
            uint32_t incl = own;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const uint32_t excl = incl - own;
            if ((int64_t)excl <= rank && rank < (int64_t)incl) {
                int64_t cum = excl;
                for (int i = 0; i < 64; i++) {
                    const uint32_t h = hist[lane * 64 + i];
                    if (rank < cum + (int64_t)h) {
                        sel[0] = lane * 64 + i;
                        sel[1] = cum;
                        break;
                    }
                    cum += h;
                }
            }
        }
        __syncthreads();
        const uint32_t b = (uint32_t)sel[0];
        rank -= sel[1];
        start += b << s;
        const uint64_t left = width - ((uint64_t)b << s);
        width = left < ((uint64_t)1 << s) ? left : ((uint64_t)1 << s);
        __syncthreads();
    }
    return start;
}

__global__ void __launch_bounds__(kRT) k_row_robust(const int32_t* __restrict__ Y, int64_t nout,
                                                    af_robust_t* __restrict__ out)
{
    __shared__ uint32_t hist[kRB];
    __shared__ long long sel[2];
    __shared__ int32_t smin[kRT / 32], smax[kRT / 32];
    const int d = blockIdx.x;
    const int32_t* y = Y + (int64_t)d * nout;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int32_t lo = INT32_MAX, hi = INT32_MIN;
    for (int64_t t = tid; t < nout; t += kRT) {
        const int32_t v = __ldg(y + t);
        lo = min(lo, v);
        hi = max(hi, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
        smin[warp] = lo;
        smax[warp] = hi;
    }
    __syncthreads();
    lo = smin[0];
    hi = smax[0];
    for (int i = 1; i < kRT / 32; i++) {
        lo = min(lo, smin[i]);
        hi = max(hi, smax[i]);
    }
    const int64_t k = (nout - 1) / 2;
    const int32_t med = lo + (int32_t)robust_select<0>(y, nout, lo, (uint32_t)(hi - lo), k, hist, sel);
    const uint32_t r2 = (uint32_t)max(hi - med, med - lo);
    const uint32_t mad = robust_select<1>(y, nout, med, r2, k, hist, sel);
    if (tid == 0) {
        out[d].median = med;
        out[d].mad = mad;
    }
}

// Robust S/N constants: snr = (B - w*med) * k, k = 1/(1.482602218505602 * mad * sqrt(w)).
__global__ void k_rowconst_robust(const af_robust_t* __restrict__ r, int ndm, af_widths_t w,
                                  af_rowconst_t* __restrict__ rc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ndm * w.n) return;
    const int d = i / w.n, wi = i % w.n;
    const int64_t W = w.w[wi];
    const double sigma = 1.482602218505602 * (double)r[d].mad;
    af_rowconst_t o;
    o.q = W * r[d].median;
    o.k = sigma > 0.0 ? (float)(1.0 / (sigma * sqrt((double)W))) : 0.0f;
    o.c = 0.0f;
    rc[(int64_t)d * AF_MAX_WIDTHS + wi] = o;
}

int launch_boxcar_tiles(const int32_t* d_plane, int ndm, int64_t nout, const af_widths_t& w,
                        const af_rowconst_t* d_rowconst, float* d_best_snr, uint8_t* d_best_w, cudaStream_t s)
{
    const unsigned tiles = (unsigned)((nout + kBOut - 1) / kBOut);
    const unsigned long long nblk = (unsigned long long)tiles * (unsigned long long)ndm;
    if (nblk > 0x7fffffffULL) return af_set_error(AF_EINVAL, "boxcar: problem too large for one grid");
    const size_t smem = (size_t)(kBOut + w.w[w.n - 1] + 1) * sizeof(uint32_t);
    if (smem > 48 * 1024)
        if (int rc = af_ensure_smem((const void*)k_boxcar, smem)) return rc;
    k_boxcar<<<(unsigned)nblk, kBT, smem, s>>>(d_plane, nout, tiles, w, d_rowconst, d_best_snr, d_best_w);
    return af_cuda_check(cudaGetLastError(), "boxcar launch");
}

}  // namespace

int af_launch_row_robust(const int32_t* d_plane, int ndm, int64_t nout, af_robust_t* d_robust, cudaStream_t s)
{
    k_row_robust<<<ndm, kRT, 0, s>>>(d_plane, nout, d_robust);
    return af_cuda_check(cudaGetLastError(), "robust row statistics launch");
}

int af_launch_boxcar_robust(const int32_t* d_plane, int ndm, int64_t nout, const af_robust_t* d_robust,
                            const af_widths_t& w, af_rowconst_t* d_rowconst, float* d_best_snr, uint8_t* d_best_w,
                            cudaStream_t s)
{
    const int nrc = ndm * w.n;
    k_rowconst_robust<<<(nrc + 255) / 256, 256, 0, s>>>(d_robust, ndm, w, d_rowconst);
    if (int rc = af_cuda_check(cudaGetLastError(), "robust rowconst launch")) return rc;
    return launch_boxcar_tiles(d_plane, ndm, nout, w, d_rowconst, d_best_snr, d_best_w, s);
}

int af_launch_boxcar(const int32_t* d_plane, int ndm, int64_t nout, const af_rowstats_t* d_stats,
                     const af_widths_t& w, af_rowconst_t* d_rowconst, float* d_best_snr, uint8_t* d_best_w,
                     cudaStream_t s)
{
    const int nrc = ndm * w.n;
    k_rowconst<<<(nrc + 255) / 256, 256, 0, s>>>(d_stats, ndm, nout, w, d_rowconst);
    if (int rc = af_cuda_check(cudaGetLastError(), "rowconst launch")) return rc;
    return launch_boxcar_tiles(d_plane, ndm, nout, w, d_rowconst, d_best_snr, d_best_w, s);
}
