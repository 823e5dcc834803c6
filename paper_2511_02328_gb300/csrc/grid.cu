// grid.cu -- DM-time slice gridding for an image detector (Sec. 2.4,
// "Griding and Rendering"): the plane's time axis is cut into slices of ns
// columns, each slice resampled to an M x M image and normalised to 8 bits.
//
//   area path (ndm > M and slice width w > M): exact pixel-area mean,
//     W(i,j) = sum_r sum_c ovr(i,r) ovc(j,c) X[r][c0 + c]   (int64, exact),
//     ovr(i,r) = |[i ndm, (i+1) ndm) & [r M, (r+1) M)|, ovc likewise with w;
//     U = W / (ndm w).
//   Lanczos-4 path otherwise: separable, source x = (i + 0.5) n / M - 0.5, taps
//     floor(x) - 3 .. floor(x) + 4, L(t) = sinc(t) sinc(t/4) normalised,
//     replicated border; evaluated in double.
//   Y = floor(255 (U - umin) / (umax - umin + eps) + 1/2), eps = 1e-6, on the
//     Lanczos path; on the area path exactly from the integers W, without eps
//     (0 for a constant slice).
//
// Two passes over the plane: the first finds each slice's min and max
// (block reduction + 64-bit atomics into the caller's work array), the
// second recomputes the values and writes Y.  One block per output row of a
// slice; a thread per output column (strided).
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace {

constexpr int kGT = 256;

// Monotone int64 key of a double (for atomic min / max).
__device__ __forceinline__ long long dkey(double v)
{
    const long long b = __double_as_longlong(v);
    return b >= 0 ? b : b ^ 0x7FFFFFFFFFFFFFFFLL;
}
__device__ __forceinline__ double dval(long long k)
{
    return __longlong_as_double(k >= 0 ? k : k ^ 0x7FFFFFFFFFFFFFFFLL);
}

__device__ __forceinline__ long long area_value(const int32_t* __restrict__ X, int64_t nout, int h, int64_t c0,
                                                int w, int M, int i, int j)
{
    const long long ri0 = (long long)i * h, ri1 = (long long)(i + 1) * h;
    const long long cj0 = (long long)j * w, cj1 = (long long)(j + 1) * w;
    const int r_lo = (int)(ri0 / M), r_hi = (int)((ri1 - 1) / M);
    const int c_lo = (int)(cj0 / M), c_hi = (int)((cj1 - 1) / M);
    long long W = 0;
    for (int r = r_lo; r <= r_hi; r++) {
        const long long ovr = min(ri1, (long long)(r + 1) * M) - max(ri0, (long long)r * M);
        const int32_t* x = X + (int64_t)r * nout + c0;
        long long row = 0;
        for (int c = c_lo; c <= c_hi; c++) {
            const long long ovc = min(cj1, (long long)(c + 1) * M) - max(cj0, (long long)c * M);
            row += ovc * (long long)__ldg(x + c);
        }
        W += ovr * row;
    }
    return W;
}

// Lanczos-4 taps of output index i for an axis of n input samples.
__device__ __forceinline__ int lanczos_taps(int i, int n, int M, double* wt)
{
    const double x = ((double)i + 0.5) * (double)n / (double)M - 0.5;
    const int k0 = (int)floor(x);
    double tot = 0.0;
#pragma unroll
    for (int a = 0; a < 8; a++) {
        const double t = x - (double)(k0 - 3 + a);
        double v;
        if (t == 0.0) {
            v = 1.0;
        } else {
            const double pt = 3.141592653589793 * t;
            v = (sinpi(t) / pt) * (sinpi(t * 0.25) / (pt * 0.25));
        }
        wt[a] = v;
        tot += v;
    }
#pragma unroll
    for (int a = 0; a < 8; a++) wt[a] /= tot;
    return k0 - 3;
}

__device__ __forceinline__ double lanczos_value(const int32_t* __restrict__ X, int64_t nout, int h, int64_t c0,
                                                int w, int M, const double* wr, int r0, int j)
{
    double wc[8];
    const int k0 = lanczos_taps(j, w, M, wc);
    double U = 0.0;
#pragma unroll
    for (int a = 0; a < 8; a++) {
        const int r = min(max(r0 + a, 0), h - 1);
        const int32_t* x = X + (int64_t)r * nout + c0;
        double row = 0.0;
#pragma unroll
        for (int b = 0; b < 8; b++) row += wc[b] * (double)__ldg(x + min(max(k0 + b, 0), w - 1));
        U += wr[a] * row;
    }
    return U;
}

__global__ void k_grid_init(long long* work, int S)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) {
        work[2 * s] = LLONG_MAX;
        work[2 * s + 1] = LLONG_MIN;
    }
}

// Block (slice s0 + blockIdx.x / M, row i = blockIdx.x % M).  PASS 0: min/max
// into work; PASS 1: write Y.
template <bool AREA, int PASS>
__global__ void __launch_bounds__(kGT) k_grid(const int32_t* __restrict__ X, int h, int64_t nout, int64_t ns, int s0,
                                              int M, long long* __restrict__ work, uint8_t* __restrict__ out)
{
    __shared__ long long slo[kGT / 32], shi[kGT / 32];
    const int s = s0 + (int)(blockIdx.x / M), i = (int)(blockIdx.x % M);
    const int64_t c0 = (int64_t)s * ns;
    const int w = (int)min(ns, nout - c0);
    double wr[8];
    int r0 = 0;
    if (!AREA) r0 = lanczos_taps(i, h, M, wr);
    if (PASS == 0) {
        long long lo = LLONG_MAX, hi = LLONG_MIN;
        for (int j = threadIdx.x; j < M; j += kGT) {
            const long long k = AREA ? area_value(X, nout, h, c0, w, M, i, j)
                                     : dkey(lanczos_value(X, nout, h, c0, w, M, wr, r0, j));
            lo = min(lo, k);
            hi = max(hi, k);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if ((threadIdx.x & 31) == 0) {
            slo[threadIdx.x >> 5] = lo;
            shi[threadIdx.x >> 5] = hi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < kGT / 32; k++) {
                lo = min(lo, slo[k]);
                hi = max(hi, shi[k]);
            }
            lo = min(lo, slo[0]);
            hi = max(hi, shi[0]);
            atomicMin(work + 2 * s, lo);
            atomicMax(work + 2 * s + 1, hi);
        }
        return;
    }
    uint8_t* o = out + ((int64_t)s * M + i) * M;
    if (AREA) {
        const long long lo = work[2 * s], hi = work[2 * s + 1];
        const unsigned long long rng = (unsigned long long)(hi - lo);
        for (int j = threadIdx.x; j < M; j += kGT) {
            const long long W = area_value(X, nout, h, c0, w, M, i, j);
            o[j] = rng == 0 ? (uint8_t)0
                            : (uint8_t)((510 * (unsigned __int128)(W - lo) + rng) / (2 * (unsigned __int128)rng));
        }
    } else {
        const double lo = dval(work[2 * s]), hi = dval(work[2 * s + 1]);
        for (int j = threadIdx.x; j < M; j += kGT) {
            const double U = lanczos_value(X, nout, h, c0, w, M, wr, r0, j);
            o[j] = (uint8_t)floor(255.0 * (U - lo) / (hi - lo + 1e-6) + 0.5);
        }
    }
}

template <int PASS>
void launch_pass(bool area, unsigned blocks, cudaStream_t st, const int32_t* X, int h, int64_t nout, int64_t ns,
                 int s0, int M, long long* work, uint8_t* out)
{
    if (area)
        k_grid<true, PASS><<<blocks, kGT, 0, st>>>(X, h, nout, ns, s0, M, work, out);
    else
        k_grid<false, PASS><<<blocks, kGT, 0, st>>>(X, h, nout, ns, s0, M, work, out);
}

}  // namespace

extern "C" int af_grid(const int32_t* d_plane, int ndm, int64_t nout, int64_t ns, int M, uint8_t* d_out,
                       int64_t* d_work, void* stream)
try {
    if (!d_plane || !d_out || !d_work) return af_set_error(AF_EINVAL, "af_grid: NULL buffer");
    if (ndm < 1 || nout < 1 || ns < 1) return af_set_error(AF_EINVAL, "af_grid: empty plane or slice");
    if (M < 2 || M > 4096) return af_set_error(AF_EINVAL, "af_grid: M %d not in 2..4096", M);
    if (ns > INT32_MAX) return af_set_error(AF_EINVAL, "af_grid: slice too long");
    // exact area sums: |W| <= ndm * ns * 2^31 must stay below 2^63
    if ((double)ndm * (double)ns * 2147483648.0 >= 9.2e18)
        return af_set_error(AF_EINVAL, "af_grid: slices of %d x %lld values are too large for exact 64-bit sums", ndm,
                            (long long)ns);
    const int64_t S = (nout + ns - 1) / ns;
    if (S * M > 0x7fffffffLL) return af_set_error(AF_EINVAL, "af_grid: too many slices");
    cudaStream_t st = (cudaStream_t)stream;
    long long* work = reinterpret_cast<long long*>(d_work);
    k_grid_init<<<(unsigned)((S + 255) / 256), 256, 0, st>>>(work, (int)S);
    if (int rc = af_cuda_check(cudaGetLastError(), "af_grid init")) return rc;
    // full slices share one path; a shorter last slice may take the other
    const int64_t nfull = nout / ns;
    const int64_t last_w = nout - nfull * ns;
    const bool area_full = ndm > M && ns > M;
    const bool area_last = ndm > M && last_w > M;
    for (int pass = 0; pass < 2; pass++) {
        if (nfull > 0) {
            if (pass == 0)
                launch_pass<0>(area_full, (unsigned)(nfull * M), st, d_plane, ndm, nout, ns, 0, M, work, d_out);
            else
                launch_pass<1>(area_full, (unsigned)(nfull * M), st, d_plane, ndm, nout, ns, 0, M, work, d_out);
        }
        if (last_w > 0) {
            if (pass == 0)
                launch_pass<0>(area_last, (unsigned)M, st, d_plane, ndm, nout, ns, (int)nfull, M, work, d_out);
            else
                launch_pass<1>(area_last, (unsigned)M, st, d_plane, ndm, nout, ns, (int)nfull, M, work, d_out);
        }
        if (int rc = af_cuda_check(cudaGetLastError(), "af_grid launch")) return rc;
    }
    return AF_OK;
} catch (...) {
    return af_host_exception("af_grid");
}
