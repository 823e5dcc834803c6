// diag.cu -- measured integer issue rates of the device, the denominator of
// the dedispersion roofline (no counterpart in the paper).
//
// Three probe kernels, one block of 1024 threads per SM (120 KB of dynamic
// shared memory keeps it to one), a fixed number of iterations each:
//   ADD:     8 independent chains of 2-input 32-bit additions per thread;
//   PATTERN: the tile kernel's inner step -- two 32-bit shared loads (two
//            channels, 4 samples each), widening into 16-bit lanes
//            (w & 0x00FF00FF, prmt(w, 0x4341)) and the paired adds -- counted
//            as 8 sample additions per iteration;
//   SHARED:  8 independent 32-bit shared loads per iteration at immediate
//            offsets from one moving base (lane-consecutive words: no bank
//            conflicts), each folded into an accumulator -- the shared-memory
//            load bandwidth the group-row tile kernel is bound by.
// Results go to a static device array (no allocation); every shared address is
// inside the block's own array.
//
// A fourth probe exercises the failure path of the bounded mbarrier waits that
// the ring kernels (tile, group-row and subband stage-2 kernels) use: one block
// waits on a barrier that nothing arrives at, with the same poll loop
// (afptx::mbar_wait_bounded), raises the error flag the way those kernels do
// and returns, so that the host reads AF_ETIMEOUT and the context stays usable.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "ptx.cuh"

namespace {

constexpr int kDT = 1024;
constexpr int kDIters = 4096;
constexpr int kDMaxBlocks = 1024;
constexpr int kDSmem = 120 * 1024;

__device__ uint32_t g_diag_sink[kDMaxBlocks];

template <int OP>
__global__ void __launch_bounds__(kDT, 1) k_diag(uint32_t seed, uint32_t mask)
{
    extern __shared__ uint32_t sm[];
    const int tid = threadIdx.x;
    for (int i = tid; i < kDSmem / 4; i += kDT) sm[i] = (uint32_t)i * 2654435761u + seed;
    __syncthreads();
    uint32_t a0 = tid ^ seed, a1 = a0 * 3u, a2 = a0 * 5u, a3 = a0 * 7u, a4 = a0 * 11u, a5 = a0 * 13u, a6 = a0 * 17u,
             a7 = a0 * 19u;
    // per warp a 2 KB slice; offsets below stay under (31 * 2048 + mask + 128) bytes < kDSmem
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm) + (tid >> 5) * 2048u + (tid & 31) * 4u;
#pragma unroll 2
    for (int it = 0; it < kDIters; it++) {
        if (OP == 0) {
            asm volatile("add.u32 %0, %0, %1;" : "+r"(a0) : "r"(a1));
            asm volatile("add.u32 %0, %0, %1;" : "+r"(a1) : "r"(a2));
            asm volatile("add.u32 %0, %0, %1;" : "+r"(a2) : "r"(a3));
            asm volatile("add.u32 %0, %0, %1;" : "+r"(a3) : "r"(a4));
            asm volatile("add.u32 %0, %0, %1;" : "+r"(a4) : "r"(a5));
            asm volatile("add.u32 %0, %0, %1;" : "+r"(a5) : "r"(a6));
            asm volatile("add.u32 %0, %0, %1;" : "+r"(a6) : "r"(a7));
            asm volatile("add.u32 %0, %0, %1;" : "+r"(a7) : "r"(a0));
        } else if (OP == 2) {
            // base + 7 * 256 + 4 stays under (31 * 2048 + mask + 1796) bytes < kDSmem
            const uint32_t b = sbase + (((uint32_t)it * 128u) & mask);
            uint32_t w0, w1, w2, w3, w4, w5, w6, w7;
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(w0) : "r"(b));
            asm volatile("ld.shared.u32 %0, [%1+256];" : "=r"(w1) : "r"(b));
            asm volatile("ld.shared.u32 %0, [%1+512];" : "=r"(w2) : "r"(b));
            asm volatile("ld.shared.u32 %0, [%1+768];" : "=r"(w3) : "r"(b));
            asm volatile("ld.shared.u32 %0, [%1+1024];" : "=r"(w4) : "r"(b));
            asm volatile("ld.shared.u32 %0, [%1+1280];" : "=r"(w5) : "r"(b));
            asm volatile("ld.shared.u32 %0, [%1+1536];" : "=r"(w6) : "r"(b));
            asm volatile("ld.shared.u32 %0, [%1+1792];" : "=r"(w7) : "r"(b));
            a0 += w0;
            a1 += w1;
            a2 += w2;
            a3 += w3;
            a4 += w4;
            a5 += w5;
            a6 += w6;
            a7 += w7;
        } else {
            // two independent accumulator pairs, one per parity of the iteration
            uint32_t w1, w2;
            const uint32_t off = ((uint32_t)it * 128u) & mask;
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(w1) : "r"(sbase + off));
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(w2) : "r"(sbase + ((off + 4096u) & mask)));
            if (it & 1) {
                a0 += (w1 & 0x00FF00FFu) + (w2 & 0x00FF00FFu);
                a1 += __byte_perm(w1, 0u, 0x4341) + __byte_perm(w2, 0u, 0x4341);
            } else {
                a2 += (w1 & 0x00FF00FFu) + (w2 & 0x00FF00FFu);
                a3 += __byte_perm(w1, 0u, 0x4341) + __byte_perm(w2, 0u, 0x4341);
            }
        }
    }
    if (tid == 0) g_diag_sink[blockIdx.x] = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7;
}

template <int OP>
int time_probe(int nblk, float* ms)
{
    if (int rc = af_ensure_smem((const void*)k_diag<OP>, kDSmem)) return rc;
    k_diag<OP><<<nblk, kDT, kDSmem>>>(12345u, 0x7fffu);
    cudaEvent_t a, b;
    AF_CUDA(cudaEventCreate(&a));
    AF_CUDA(cudaEventCreate(&b));
    cudaEventRecord(a);
    k_diag<OP><<<nblk, kDT, kDSmem>>>(777u, 0x7fffu);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return af_cuda_check(e, "af_diag_int_rates probe");
}

// Error flag of the bounded-wait probe (a static device variable: no allocation).
__device__ int g_diag_wait_err;

// One block of 128 threads waits on an mbarrier of one arrival.  arrive = 1:
// thread 0 arrives, the phase completes and every wait succeeds.  arrive = 0:
// nothing arrives, every thread's wait gives up after `polls` polls, lane 0 of
// each warp raises the flag (as the ring kernels' warps do) and the block
// returns.  No copy is in flight, so nothing else has to drain.
__global__ void __launch_bounds__(128) k_diag_wait(int arrive, uint32_t polls)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = afptx::smem_addr(&bar);
    if (threadIdx.x == 0) {
        afptx::mbar_init(b, 1);
        afptx::fence_mbar_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0) afptx::mbar_arrive(b);
    if (!afptx::mbar_wait_bounded(b, 0u, polls) && (threadIdx.x & 31) == 0) atomicExch(&g_diag_wait_err, 1);
    __syncthreads();
    if (threadIdx.x == 0) afptx::mbar_inval(b);
}

}  // namespace

extern "C" int af_diag_smem_rate(double* bytes_per_s)
try {
    if (!bytes_per_s) return af_set_error(AF_EINVAL, "af_diag_smem_rate: NULL output");
    int dev = 0, nsm = 0;
    AF_CUDA(cudaGetDevice(&dev));
    AF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int nblk = nsm < kDMaxBlocks ? nsm : kDMaxBlocks;
    float ms = 0.f;
    if (int rc = time_probe<2>(nblk, &ms)) return rc;
    *bytes_per_s = (double)nblk * kDT * kDIters * 8.0 * 4.0 / (ms * 1e-3);
    return AF_OK;
} catch (...) {
    return af_host_exception("af_diag_smem_rate");
}

extern "C" int af_diag_int_rates(double* add_per_s, double* pattern_adds_per_s)
try {
    if (!add_per_s || !pattern_adds_per_s) return af_set_error(AF_EINVAL, "af_diag_int_rates: NULL output");
    int dev = 0, nsm = 0;
    AF_CUDA(cudaGetDevice(&dev));
    AF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int nblk = nsm < kDMaxBlocks ? nsm : kDMaxBlocks;
    float ms0 = 0.f, ms1 = 0.f;
    if (int rc = time_probe<0>(nblk, &ms0)) return rc;
    if (int rc = time_probe<1>(nblk, &ms1)) return rc;
    const double threads = (double)nblk * kDT * kDIters;
    *add_per_s = threads * 8.0 / (ms0 * 1e-3);
    *pattern_adds_per_s = threads * 8.0 / (ms1 * 1e-3);
    return AF_OK;
} catch (...) {
    return af_host_exception("af_diag_int_rates");
}

extern "C" int af_diag_bounded_wait(int arrive, int64_t polls, float* ms)
try {
    if (polls < 1 || polls > (int64_t)1 << 24)
        return af_set_error(AF_EINVAL, "af_diag_bounded_wait: polls %lld outside 1..2^24", (long long)polls);
    const int zero = 0;
    AF_CUDA(cudaMemcpyToSymbol(g_diag_wait_err, &zero, sizeof zero));
    cudaEvent_t a, b;
    AF_CUDA(cudaEventCreate(&a));
    AF_CUDA(cudaEventCreate(&b));
    cudaEventRecord(a);
    k_diag_wait<<<1, 128>>>(arrive ? 1 : 0, (uint32_t)polls);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&err, g_diag_wait_err, sizeof err);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (int rc = af_cuda_check(e, "af_diag_bounded_wait")) return rc;
    if (ms) *ms = t;
    if (err)
        return af_set_error(AF_ETIMEOUT, "af_diag_bounded_wait: the wait ran out after %lld polls (%.3f ms)",
                            (long long)polls, (double)t);
    return AF_OK;
} catch (...) {
    return af_host_exception("af_diag_bounded_wait");
}
