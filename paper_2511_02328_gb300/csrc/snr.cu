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
constexpr int kPer = 16;             // outputs per thread
constexpr int kBOut = kBT * kPer;    // outputs per block

// Block = one tile of kBOut outputs of one row.
//  1. Y[t0 .. t0 + L), L = kBOut + wmax - 1 (clipped at nout), is loaded into
//     shared memory with coalesced (16-byte when aligned) loads, all issued
//     before any is used.
//  2. Prefix sums P[j] = sum_{k<j} Y[t0+k] (mod 2^32) in one pass: thread i
//     scans its own segment of C consecutive values (C odd, so a warp's
//     segment accesses fall in distinct banks), the segment totals are scanned
//     across the block, and each thread adds its offset.
//  3. Output t0 + lt (lt = tid + kBT*i) evaluates every width from P[lt] and
//     P[lt + w]: B = P[lt+w] - P[lt], snr = (B - q) * k - c.
// With SMALL (every window sum < 2^31) the difference B - q is formed and
// converted in 32 bits.
template <bool SMALL>
__global__ void __launch_bounds__(kBT, 4)
k_boxcar(const int32_t* __restrict__ Y, int64_t nout, unsigned tiles, af_widths_t w,
         const af_rowconst_t* __restrict__ rc, float* __restrict__ snr, uint8_t* __restrict__ bw)
{
    extern __shared__ uint32_t sP[];  // 3 words of padding, then P[0 .. kBT*C]
    __shared__ int64_t sq[AF_MAX_WIDTHS];
    __shared__ float sk[AF_MAX_WIDTHS], sc[AF_MAX_WIDTHS];
    __shared__ int sw[AF_MAX_WIDTHS];
    __shared__ uint32_t swarp[kBT / 32];
    uint32_t* P = sP + 3;             // P[1 + j] holds Y[t0 + j]: 16-byte aligned for j % 4 == 0

    const int d = (int)(blockIdx.x / tiles);
    const int64_t t0 = (int64_t)(blockIdx.x % tiles) * kBOut;
    const int nw = w.n;
    const int wmax = w.w[nw - 1];
    const int L = (int)(min(nout, t0 + kBOut + wmax - 1) - t0);
    const int64_t base = (int64_t)d * nout + t0;
    const int32_t* y = Y + base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid < nw) {
        const af_rowconst_t c = rc[(int64_t)d * AF_MAX_WIDTHS + tid];
        sq[tid] = c.q;
        sk[tid] = c.k;
        sc[tid] = c.c;
        sw[tid] = w.w[tid];
    }
    // 1. load Y into P[1 .. L]
    int done = 0;
    if ((reinterpret_cast<uintptr_t>(y) & 15) == 0) {
        // every load of the tile is issued before the first shared store
        constexpr int NB = (kBOut + 1024) / 4 / kBT;  // 16-byte loads per thread (L <= kBOut + 1023)
        const int L4 = L >> 2;
        const int4* y4 = reinterpret_cast<const int4*>(y);
        int4 v[NB];
#pragma unroll
        for (int u = 0; u < NB; u++)
            if (tid + u * kBT < L4) v[u] = __ldg(y4 + tid + u * kBT);
#pragma unroll
        for (int u = 0; u < NB; u++)
            if (tid + u * kBT < L4) reinterpret_cast<int4*>(P + 1)[tid + u * kBT] = v[u];
        for (int j = tid + NB * kBT; j < L4; j += kBT) reinterpret_cast<int4*>(P + 1)[j] = __ldg(y4 + j);
        done = 4 * L4;
    }
    for (int j = done + tid; j < L; j += kBT) P[j + 1] = (uint32_t)__ldg(y + j);
    const int C = ((L + kBT - 1) / kBT) | 1;
    for (int j = L + 1 + tid; j <= kBT * C; j += kBT) P[j] = 0u;  // pad the last segments
    if (tid == 0) P[0] = 0u;
    __syncthreads();

    // 2. prefix sums: the segment of thread tid is P[1 + tid*C .. 1 + (tid+1)*C)
    uint32_t* seg = P + 1 + tid * C;
    uint32_t run = 0;
    for (int k = 0; k < C; k++) {
        run += seg[k];
        seg[k] = run;
    }
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) swarp[warp] = incl;
    __syncthreads();
    uint32_t off = incl - run;
    for (int k = 0; k < warp; k++) off += swarp[k];
    for (int k = 0; k < C; k++) seg[k] += off;
    __syncthreads();

    // 3. S/N of every width, best width.  Tiles whose every window ends
    //    inside the row take the unchecked path: widths outer, the thread's
    //    kPer outputs inner (independent chains).
    if (t0 + kBOut + wmax - 1 <= nout) {
        uint32_t p0[kPer];
        float best[kPer];
        int bi[kPer];
#pragma unroll
        for (int i = 0; i < kPer; i++) {
            p0[i] = P[i * kBT + tid];
            best[i] = -INFINITY;
            bi[i] = AF_NO_WIDTH;
        }
        for (int k = 0; k < nw; k++) {
            const int ww = sw[k];
            const float kk = sk[k], cc = -sc[k];
            const int64_t qq = sq[k];
#pragma unroll
            for (int i = 0; i < kPer; i++) {
                const uint32_t B = P[i * kBT + tid + ww] - p0[i];
                float x;
                if (SMALL)
                    x = (float)((int32_t)B - (int32_t)qq);
                else
                    x = (float)((int64_t)B - qq);
                const float v = fmaf(x, kk, cc);
                if (v > best[i]) {
                    best[i] = v;
                    bi[i] = k;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kPer; i++) {
            const int64_t o = base + i * kBT + tid;
            snr[o] = best[i];
            if (bw) bw[o] = (uint8_t)bi[i];
        }
        return;
    }
#pragma unroll 1
    for (int i = 0; i < kPer; i++) {
        const int lt = i * kBT + tid;
        const int64_t t = t0 + lt;
        if (t >= nout) break;
        const uint32_t p0 = P[lt];
        float best = -INFINITY;
        int bi = AF_NO_WIDTH;
        for (int k = 0; k < nw; k++) {
            const int ww = sw[k];
            if (t + ww > nout) break;
            const uint32_t B = P[lt + ww] - p0;
            float x;
            if (SMALL)
                x = (float)((int32_t)B - (int32_t)sq[k]);
            else
                x = (float)((int64_t)B - sq[k]);
            const float v = fmaf(x, sk[k], -sc[k]);
            if (v > best) {
                best = v;
                bi = k;
            }
        }
        const int64_t o = base + lt;
        snr[o] = best;
        if (bw) bw[o] = (uint8_t)bi;
    }
}

int launch_boxcar_tiles(const int32_t* d_plane, int ndm, int64_t nout, const af_widths_t& w,
                        const af_rowconst_t* d_rowconst, float* d_best_snr, uint8_t* d_best_w, cudaStream_t s)
{
    const unsigned tiles = (unsigned)((nout + kBOut - 1) / kBOut);
    const unsigned long long nblk = (unsigned long long)tiles * (unsigned long long)ndm;
    if (nblk > 0x7fffffffULL) return af_set_error(AF_EINVAL, "boxcar: problem too large for one grid");
    const int L = kBOut + w.w[w.n - 1] - 1;
    const int C = ((L + kBT - 1) / kBT) | 1;
    const size_t smem = (size_t)(kBT * C + 4) * sizeof(uint32_t);
    const void* fn = w.small ? (const void*)k_boxcar<true> : (const void*)k_boxcar<false>;
    if (smem > 48 * 1024)
        if (int rc = af_ensure_smem(fn, smem)) return rc;
    if (w.small)
        k_boxcar<true><<<(unsigned)nblk, kBT, smem, s>>>(d_plane, nout, tiles, w, d_rowconst, d_best_snr, d_best_w);
    else
        k_boxcar<false><<<(unsigned)nblk, kBT, smem, s>>>(d_plane, nout, tiles, w, d_rowconst, d_best_snr, d_best_w);
    return af_cuda_check(cudaGetLastError(), "boxcar launch");
}

// ---------------------------------------------------------------- robust S/N
// Per-row median and MAD (lower medians, exact) by radix selection: one block
// per row; each pass histograms a window of the value range into at most 2048
// bins in shared memory and keeps the bin holding the wanted rank, so a window
// of R values takes ceil(log2(R) / 11) passes.
//
// Windows.  A first pass takes the row's minimum, maximum, mean mu and a bound
// s >= sigma on its standard deviation.  Any median m of a distribution lies
// within sigma of its mean (Cantelli), so the median is searched in
// [mu - s - 1, mu + s + 1]; and since E|X - m| <= E|X - mu| <= sigma, Markov's
// inequality leaves at most half of the values at |X - m| >= 2 sigma, so the
// lower median of |X - m| (the MAD) is below 2 sigma and is searched in
// [0, 2 s + 1].  For noise-like rows both windows are under 2048 wide: one
// pass each, three passes in all (five over the full ranges).  The first
// histogram pass of each search also counts the values below its window and
// in it; the selection goes on only if the wanted rank falls inside, which
// makes the result exact whatever the floating-point bound -- otherwise (never
// expected) the same selection runs on the full range.
constexpr int kRT = 512;
constexpr int kRB = 2048;

template <int MODE>  // 0: u = v - base;  1: u = |v - base|   (mod 2^32, no signed overflow)
__device__ __forceinline__ uint32_t robust_key(int32_t v, int32_t base)
{
    if (MODE == 0) return (uint32_t)v - (uint32_t)base;
    return v >= base ? (uint32_t)v - (uint32_t)base : (uint32_t)base - (uint32_t)v;
}

// Calls f(v) for every value of the row y[0 .. n), spread over the block: a
// scalar head up to the first 16-byte boundary, then kRU4 16-byte loads per
// thread in flight per step, then the scalar tail.
constexpr int kRU4 = 4;
template <typename F>
__device__ __forceinline__ void for_row(const int32_t* __restrict__ y, int64_t n, F&& f)
{
    const int tid = threadIdx.x;
    int64_t head = (int64_t)(((16u - ((uint32_t)reinterpret_cast<uintptr_t>(y) & 15u)) & 15u) >> 2);
    if (head > n) head = n;
    if (tid < head) f(__ldg(y + tid));
    const int4* y4 = reinterpret_cast<const int4*>(y + head);
    const int64_t n4 = (n - head) >> 2;
    for (int64_t i = tid; i < n4; i += (int64_t)kRT * kRU4) {
        int4 v[kRU4];
#pragma unroll
        for (int u = 0; u < kRU4; u++)
            if (i + u * kRT < n4) v[u] = __ldg(y4 + i + u * kRT);
#pragma unroll
        for (int u = 0; u < kRU4; u++)
            if (i + u * kRT < n4) {
                f(v[u].x);
                f(v[u].y);
                f(v[u].z);
                f(v[u].w);
            }
    }
    const int64_t t0 = head + 4 * n4;
    if (t0 + tid < n) f(__ldg(y + t0 + tid));  // at most 3 values
}

// Block sum of one int64 per thread, returned to every thread (sred: kRT/32 slots).
__device__ __forceinline__ long long block_sum(long long x, long long* sred)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();  // earlier readers of sred are done
    if (lane == 0) sred[warp] = x;
    __syncthreads();
    long long t = 0;
    for (int i = 0; i < kRT / 32; i++) t += sred[i];
    return t;
}

// The rank-th smallest key (0-based) among the row's keys in [0, width).  For
// MODE 0, rank counts from the row's smallest value: the first pass counts
// the values under `base` (none when base is the row minimum).  Returns false,
// with every thread agreeing, when the first pass shows the rank outside the
// window.
template <int MODE>
__device__ bool robust_select(const int32_t* __restrict__ y, int64_t n, int32_t base, uint64_t width, int64_t rank,
                              uint32_t* hist, long long* sel, long long* sred, uint32_t* out)
{
    uint32_t start = 0;
    const int tid = threadIdx.x, lane = tid & 31;
    bool first = true;
    while (first || width > 1) {
        const int bits = width > 1 ? 64 - __clzll((long long)(width - 1)) : 0;
        const int s = bits > 11 ? bits - 11 : 0;
        for (int i = tid; i < kRB; i += kRT) hist[i] = 0u;
        __syncthreads();
        long long below = 0;
        const bool count_below = MODE == 0 && first;
        for_row(y, n, [&](int32_t v) {
            const uint32_t k = robust_key<MODE>(v, base);
            if (k >= start && (uint64_t)(k - start) < width) atomicAdd(&hist[(k - start) >> s], 1u);
            else if (count_below && v < base) below++;
        });
        if (MODE == 0 && first) rank -= block_sum(below, sred);  // syncs the block
        else __syncthreads();
        if (tid < 32) {
            // lane l owns bins [64 l, 64 l + 64): find the bin where the count passes rank
            uint32_t own = 0;
#pragma unroll 8
            for (int i = 0; i < 64; i++) own += hist[lane * 64 + i];
            uint32_t incl = own;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            if (lane == 0) sel[2] = (rank >= 0 && rank < (int64_t)total) ? 1 : 0;
            const uint32_t excl = incl - own;
            if ((int64_t)excl <= rank && rank < (int64_t)incl) {
                int64_t cum = excl;
#pragma unroll 1
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
        if (!sel[2]) return false;  // only on a first pass: later windows hold the rank by construction
        const uint32_t b = (uint32_t)sel[0];
        rank -= sel[1];
        start += b << s;
        const uint64_t left = width - ((uint64_t)b << s);
        width = left < ((uint64_t)1 << s) ? left : ((uint64_t)1 << s);
        first = false;
        __syncthreads();
    }
    *out = start;
    return true;
}

__global__ void __launch_bounds__(kRT, 2) k_row_robust(const int32_t* __restrict__ Y, int64_t nout,
                                                    af_robust_t* __restrict__ out)
{
    __shared__ uint32_t hist[kRB];
    __shared__ long long sel[3];
    __shared__ long long sred[kRT / 32];
    __shared__ int32_t smin[kRT / 32], smax[kRT / 32];
    __shared__ float ssq[kRT / 32];
    const int d = blockIdx.x;
    const int32_t* y = Y + (int64_t)d * nout;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // pass 1: range, and sums of u = v - y[0] (exact) and of u^2 (fp32 per thread; only the window depends on it)
    const int32_t y0 = __ldg(y);
    int32_t lo = INT32_MAX, hi = INT32_MIN;
    long long su = 0;
    float sq = 0.0f;
    for_row(y, nout, [&](int32_t v) {
        lo = min(lo, v);
        hi = max(hi, v);
        su += (long long)v - y0;
        // v - y0 mod 2^32 as a signed value: exact unless the row spans more
        // than 2^31, where only the window estimate (never the result) suffers
        const float f = (float)(int32_t)((uint32_t)v - (uint32_t)y0);
        sq = fmaf(f, f, sq);
    });
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
    }
    if (lane == 0) {
        smin[warp] = lo;
        smax[warp] = hi;
        ssq[warp] = sq;
    }
    su = block_sum(su, sred);  // syncs: smin, smax, ssq are visible
    lo = smin[0];
    hi = smax[0];
    double m2 = 0.0;
    for (int i = 0; i < kRT / 32; i++) {
        lo = min(lo, smin[i]);
        hi = max(hi, smax[i]);
        m2 += (double)ssq[i];
    }
    const double nn = (double)nout, mean_u = (double)su / nn;
    m2 /= nn;
    // s >= sigma: the fp32 sums of u^2 (about nout / 512 terms per thread, then 32
    // per warp) carry a relative error below (terms) * 2^-24; the margin is 4x that
    const double rel = 1e-4 + ((double)nout / kRT + 64.0) * 2.4e-7;
    const double sb = sqrt(fmax(m2 - mean_u * mean_u, 0.0) + rel * m2 + 1.0);
    const double mu = (double)y0 + mean_u;
    const int64_t k = (nout - 1) / 2;

    const int64_t wl = max((int64_t)lo, (int64_t)floor(mu - sb) - 1);
    const int64_t wh = min((int64_t)hi, (int64_t)ceil(mu + sb) + 1);
    uint32_t key = 0;
    int32_t med;
    if (wl <= wh && robust_select<0>(y, nout, (int32_t)wl, (uint64_t)(wh - wl) + 1, k, hist, sel, sred, &key))
        med = (int32_t)((uint32_t)(int32_t)wl + key);  // a row value: no overflow in the sum
    else {  // the same selection over the whole range [lo, hi]
        robust_select<0>(y, nout, lo, (uint64_t)((int64_t)hi - lo) + 1, k, hist, sel, sred, &key);
        med = (int32_t)((uint32_t)lo + key);
    }
    const int64_t r2 = max((int64_t)hi - med, (int64_t)med - lo);
    const int64_t wm = min(r2, (int64_t)ceil(2.0 * sb) + 1);
    uint32_t mad = 0;
    if (!robust_select<1>(y, nout, med, (uint64_t)wm + 1, k, hist, sel, sred, &mad))
        robust_select<1>(y, nout, med, (uint64_t)r2 + 1, k, hist, sel, sred, &mad);
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
