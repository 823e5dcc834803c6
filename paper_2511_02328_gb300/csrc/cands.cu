// cands.cu -- thresholding and compaction of S/N peaks into a candidate list
// (the S/N criterion of Sec. 2; the local-maximum rule is stated in afgb.h).
//
// One thread per (row, t).  Threads above threshold test the +-w
// neighbourhood of their own best width, then each warp appends its
// candidates with one atomic on the shared cursor (ballot + popc).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace {

constexpr int kCT = 256;

__global__ void __launch_bounds__(kCT)
k_candidates(const float* __restrict__ snr, const uint8_t* __restrict__ bw, int64_t nout, unsigned tiles,
             af_widths_t w, float thresh, int64_t sample0, af_cand_t* __restrict__ out, int32_t cap,
             int32_t* __restrict__ count)
{
    const int d = (int)(blockIdx.x / tiles);
    const int64_t t = (int64_t)(blockIdx.x % tiles) * kCT + threadIdx.x;
    const float* row = snr + (int64_t)d * nout;
    bool pred = false;
    int width = 0;
    float s = 0.0f;
    if (t < nout) {
        s = __ldg(row + t);
        if (s >= thresh) {
            const int bi = __ldg(bw + (int64_t)d * nout + t);
            if (bi < w.n) {
                width = w.w[bi];
                pred = true;
                const int64_t lo = t - width < 0 ? 0 : t - width;
                const int64_t hi = t + width > nout - 1 ? nout - 1 : t + width;
                for (int64_t u = lo; u < t && pred; u++)
                    if (!(s > __ldg(row + u))) pred = false;
                for (int64_t u = t + 1; u <= hi && pred; u++)
                    if (!(s >= __ldg(row + u))) pred = false;
            }
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    if (m == 0u) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) {
        const int idx = base + __popc(m & ((1u << lane) - 1u));
        if (idx < cap) {
            af_cand_t c;
            c.dm_idx = d;
            c.t = (int32_t)t;
            c.width = width;
            c.snr = s;
            c.abs_sample = sample0 + t;
            out[idx] = c;
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
    const unsigned tiles = (unsigned)((nout + kCT - 1) / kCT);
    const unsigned long long nblk = (unsigned long long)tiles * (unsigned long long)ndm;
    if (nblk > 0x7fffffffULL) return af_set_error(AF_EINVAL, "candidates: problem too large for one grid");
    k_candidates<<<(unsigned)nblk, kCT, 0, s>>>(d_best_snr, d_best_w, nout, tiles, w, thresh, sample0, d_out, cap,
                                                d_count);
    return af_cuda_check(cudaGetLastError(), "candidates launch");
}
