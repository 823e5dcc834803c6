// dedisp.cu -- brute-force incoherent dedispersion (Sec. 2.3) and row sums.
//
//   Y[d][t] = sum_c X[c][t + D[d][c]],  0 <= t < nout,  exact int32.
//
// First version: each thread owns one output column t of a block of DB DM
// rows and walks all channels, reading the input through the L1 cache; the
// block's delays for a chunk of 64 channels are staged in shared memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace {

constexpr int kDB = 8;        // DM rows per block
constexpr int kThreads = 256; // one output column per thread
constexpr int kCChunk = 64;   // channels whose delays are staged at a time

__global__ void __launch_bounds__(kThreads)
k_dedisp_simple(const uint8_t* __restrict__ X, int64_t nsamp, int nchan, const int32_t* __restrict__ D,
                int ndm, int64_t nout, int32_t* __restrict__ Y, unsigned tiles)
{
    __shared__ int32_t sD[kDB][kCChunk];
    // one flat grid: block b covers DM block b / tiles and time tile b % tiles
    const int d0 = (int)(blockIdx.x / tiles) * kDB;
    const int64_t t = (int64_t)(blockIdx.x % tiles) * kThreads + threadIdx.x;
    int32_t acc[kDB];
#pragma unroll
    for (int i = 0; i < kDB; i++) acc[i] = 0;
    for (int c0 = 0; c0 < nchan; c0 += kCChunk) {
        const int cn = min(kCChunk, nchan - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < kDB * kCChunk; i += kThreads) {
            const int dd = i / kCChunk, cc = i % kCChunk;
            sD[dd][cc] = (d0 + dd < ndm && cc < cn) ? D[(int64_t)(d0 + dd) * nchan + c0 + cc] : 0;
        }
        __syncthreads();
        if (t < nout) {
            for (int cc = 0; cc < cn; cc++) {
                const uint8_t* xc = X + (int64_t)(c0 + cc) * nsamp + t;
#pragma unroll
                for (int dd = 0; dd < kDB; dd++) acc[dd] += (int32_t)__ldg(xc + sD[dd][cc]);
            }
        }
    }
    if (t < nout) {
#pragma unroll
        for (int dd = 0; dd < kDB; dd++)
            if (d0 + dd < ndm) Y[(int64_t)(d0 + dd) * nout + t] = acc[dd];
    }
}

// Row sums: one block per row, int64 sum and sum of squares.
constexpr int kStatThreads = 256;

__global__ void __launch_bounds__(kStatThreads)
k_rowstats(const int32_t* __restrict__ Y, int64_t nout, af_rowstats_t* __restrict__ st)
{
    const int d = blockIdx.x;
    const int32_t* y = Y + (int64_t)d * nout;
    long long s = 0, q = 0;
    for (int64_t t = threadIdx.x; t < nout; t += kStatThreads) {
        const long long v = __ldg(y + t);
        s += v;
        q += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    __shared__ long long ss[kStatThreads / 32], sq[kStatThreads / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        ss[w] = s;
        sq[w] = q;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0, b = 0;
        for (int i = 0; i < kStatThreads / 32; i++) {
            a += ss[i];
            b += sq[i];
        }
        st[d].sum = a;
        st[d].sumsq = b;
    }
}

}  // namespace

int af_prepare_dedisp_tables(af_plan_t p)
{
    (void)p;
    return AF_OK;
}

int af_launch_dedisperse(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int64_t nout, int32_t* d_plane,
                         cudaStream_t s)
{
    const unsigned tiles = (unsigned)((nout + kThreads - 1) / kThreads);
    const unsigned long long nblk = (unsigned long long)tiles * (unsigned long long)((p->ndm + kDB - 1) / kDB);
    if (nblk > 0x7fffffffULL) return af_set_error(AF_EINVAL, "dedisperse: problem too large for one grid");
    k_dedisp_simple<<<(unsigned)nblk, kThreads, 0, s>>>(d_in, nsamp, p->nchan, p->d_delays, p->ndm, nout, d_plane,
                                                        tiles);
    return af_cuda_check(cudaGetLastError(), "dedisperse launch");
}

int af_launch_rowstats(const int32_t* d_plane, int ndm, int64_t nout, af_rowstats_t* d_stats, cudaStream_t s)
{
    k_rowstats<<<ndm, kStatThreads, 0, s>>>(d_plane, nout, d_stats);
    return af_cuda_check(cudaGetLastError(), "rowstats launch");
}
