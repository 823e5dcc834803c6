// cands.cu -- thresholding and compaction of S/N peaks into a candidate list
// (the S/N criterion of Sec. 2; the local-maximum rule is stated in afgb.h).
//
// The plane is read as one flat array of ndm*nout values, 4 consecutive values
// per thread per step (one 16-byte load when the plane is 16-byte aligned),
// in a grid-stride loop over one resident wave of blocks.  The rare values above
// threshold derive (d, t) and test the +-w neighbourhood of their own best
// width along their row; each warp appends its candidates with one atomic on
// the shared cursor per value slot (ballot + popc).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace {

constexpr int kCT = 256;
constexpr int kCU = 2;  // 4-value groups per thread per step

__device__ __forceinline__ float4 load4(const float* __restrict__ snr, int64_t g, int64_t total, bool vec)
{
    const int64_t e = 4 * g;
    if (vec && e + 3 < total) return __ldg(reinterpret_cast<const float4*>(snr) + g);
    float4 v = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
    if (e < total) v.x = __ldg(snr + e);
    if (e + 1 < total) v.y = __ldg(snr + e + 1);
    if (e + 2 < total) v.z = __ldg(snr + e + 2);
    if (e + 3 < total) v.w = __ldg(snr + e + 3);
    return v;
}

// Is flat element e (value s >= thresh) a candidate?  Sets its width.
__device__ __forceinline__ bool is_peak(const float* __restrict__ snr, const uint8_t* __restrict__ bw,
                                        int64_t nout, const af_widths_t& w, int64_t e, float s, int& width)
{
    const int bi = __ldg(bw + e);
    if (bi >= w.n) return false;
    width = w.w[bi];
    const int64_t d = e / nout, t = e - d * nout;
    const float* row = snr + d * nout;
    const int64_t lo = t - width < 0 ? 0 : t - width;
    const int64_t hi = t + width > nout - 1 ? nout - 1 : t + width;
    for (int64_t u = lo; u < t; u++)
        if (!(s > __ldg(row + u))) return false;
    for (int64_t u = t + 1; u <= hi; u++)
        if (!(s >= __ldg(row + u))) return false;
    return true;
}

__global__ void __launch_bounds__(kCT)
k_candidates(const float* __restrict__ snr, const uint8_t* __restrict__ bw, int64_t nout, int64_t total, bool vec,
             af_widths_t w, float thresh, int64_t sample0, af_cand_t* __restrict__ out, int32_t cap,
             int32_t* __restrict__ count)
{
    const int64_t ngroups = (total + 3) / 4;
    const int lane = threadIdx.x & 31;
    // every thread of a block runs the same number of steps (warp-uniform ballots)
    for (int64_t g0 = (int64_t)blockIdx.x * (kCT * kCU); g0 < ngroups; g0 += (int64_t)gridDim.x * (kCT * kCU)) {
        float4 v[kCU];
#pragma unroll
        for (int u = 0; u < kCU; u++) {
            const int64_t g = g0 + u * kCT + threadIdx.x;
            v[u] = g < ngroups ? load4(snr, g, total, vec)
                               : make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
        }
        float m = -INFINITY;
#pragma unroll
        for (int u = 0; u < kCU; u++) m = fmaxf(m, fmaxf(fmaxf(v[u].x, v[u].y), fmaxf(v[u].z, v[u].w)));
        if (!__any_sync(0xffffffffu, m >= thresh)) continue;
#pragma unroll
        for (int u = 0; u < kCU; u++) {
            const int64_t e0 = 4 * (g0 + u * kCT + threadIdx.x);
            const float sv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float s = sv[j];
                int width = 0;
                const bool pred = s >= thresh && is_peak(snr, bw, nout, w, e0 + j, s, width);
                const unsigned msk = __ballot_sync(0xffffffffu, pred);
                if (msk == 0u) continue;
                const int leader = __ffs(msk) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(count, __popc(msk));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (pred) {
                    const int idx = base + __popc(msk & ((1u << lane) - 1u));
                    if (idx < cap) {
                        const int64_t d = (e0 + j) / nout, t = e0 + j - d * nout;
                        af_cand_t c;
                        c.dm_idx = (int32_t)d;
                        c.t = (int32_t)t;
                        c.width = width;
                        c.snr = s;
                        c.abs_sample = sample0 + t;
                        out[idx] = c;
                    }
                }
            }
        }
    }
}

}  // namespace

int af_launch_candidates(const float* d_best_snr, const uint8_t* d_best_w, int ndm, int64_t nout,
                         const af_widths_t& w, float thresh, int64_t sample0, af_cand_t* d_out, int32_t cap,
                         int32_t* d_count, cudaStream_t s)
{
    if (int rc = af_cuda_check(cudaMemsetAsync(d_count, 0, sizeof(int32_t), s), "candidates count reset"))
        return rc;
    const int64_t total = (int64_t)ndm * nout;
    const int64_t steps = (total + 4LL * kCT * kCU - 1) / (4LL * kCT * kCU);
    // one resident wave: SMs x resident blocks per SM (cached per device)
    static int resident[64];
    int dev = 0;
    if (int rc = af_cuda_check(cudaGetDevice(&dev), "candidates device")) return rc;
    if (dev < 0 || dev >= 64) return af_set_error(AF_EINVAL, "candidates: device index above 63");
    if (resident[dev] == 0) {
        int nsm = 0, per = 0;
        if (int rc = af_cuda_check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count"))
            return rc;
        if (int rc = af_cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_candidates, kCT, 0),
                                   "candidates occupancy"))
            return rc;
        resident[dev] = nsm * (per > 0 ? per : 1);
    }
    const int64_t nblk = steps < resident[dev] ? (steps > 0 ? steps : 1) : resident[dev];
    const bool vec = (reinterpret_cast<uintptr_t>(d_best_snr) & 15) == 0;
    k_candidates<<<(unsigned)nblk, kCT, 0, s>>>(d_best_snr, d_best_w, nout, total, vec, w, thresh, sample0, d_out,
                                                cap, d_count);
    return af_cuda_check(cudaGetLastError(), "candidates launch");
}
