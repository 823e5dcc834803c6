// cutout.cu -- the classifier's input: two 64 x 64 cut-outs around each
// candidate (DM-time from the plane, frequency-time from the input
// dedispersed at the candidate's DM), min-max normalised and rounded to
// bfloat16.  This replaces the paper's gridding of DM-time slices into
// 512 x 512 images (Sec. 2.4) and keeps its per-image min-max normalisation
// (without the 8-bit quantisation).  Definitions, per candidate (d, t, w):
//   bins       b = max(1, w / 2); bin j covers output samples
//              [t - 32 b + j b, t - 32 b + (j + 1) b), samples outside [0, nout) count 0
//   DM-time    [i][j] = sum over the bin of plane row d - 32 + i (0 outside [0, ndm))
//   freq-time  [g][j] = sum over channels c of group g (nchan / 64 each) and the
//              bin's samples s of X[c][s + D[d][c]]
//   normalise  v' = float(v - min) / (float(max - min) + 1e-6f), then bf16 (rn)
// Output NHWC bf16 [n][64][64][2]: channel 0 DM-time, 1 freq-time.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "internal.h"
#include "nn.h"

namespace {

constexpr int S = 64, T = 512, NWARP = T / 32;
constexpr int CH = 128;  // window positions per chunk (4 per lane)
constexpr int kDelaysInShared = 8192;  // channels whose delay row is staged in shared memory

__device__ __forceinline__ void block_minmax(long long& lo, long long& hi)
{
    __shared__ long long slo[NWARP], shi[NWARP];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        slo[w] = lo;
        shi[w] = hi;
    }
    __syncthreads();
    lo = slo[0];
    hi = shi[0];
    for (int i = 1; i < NWARP; i++) {
        lo = min(lo, slo[i]);
        hi = max(hi, shi[i]);
    }
    __syncthreads();
}

// Adds the window positions of this warp's chunk [p0, p0 + CH) held in pos[]
// to the lane's two bins 2*lane, 2*lane + 1 (bin j = positions [j b, (j+1) b)).
__device__ __forceinline__ void bin_chunk(const int32_t* pos, int p0, int b, int lane, long long& b0,
                                          long long& b1)
{
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int j = 2 * lane + h;
        const int lo = max(j * b, p0), hi = min((j + 1) * b, p0 + CH);
        long long acc = 0;
        for (int p = lo; p < hi; p++) acc += pos[p - p0];
        if (h == 0)
            b0 += acc;
        else
            b1 += acc;
    }
}

// One block per candidate.  Window positions p in [0, 64 b) are samples
// start + p, start = t - 32 b; bin j holds positions [j b, (j+1) b); samples
// outside [0, nout) count 0.  Each warp owns image rows (channel groups for
// the frequency-time image, plane rows for the DM-time image); per row it
// walks the window in chunks of 128 positions, lane l reading positions
// 4l .. 4l+3 of the chunk (consecutive lanes: consecutive bytes or words),
// summing over the row's channels in registers, then folding the chunk into
// its two bins through a per-warp shared array.
__global__ void __launch_bounds__(T, 1) k_cutout(const uint8_t* __restrict__ X, int64_t nsamp, int nchan,
                                              const int32_t* __restrict__ D, int ndm,
                                              const int32_t* __restrict__ plane, int64_t nout,
                                              const af_cand_t* __restrict__ cands, __nv_bfloat16* __restrict__ out)
{
    __shared__ int32_t pos[NWARP][CH];  // a chunk's column sums (plane values, or <= 255 * 1024)
    __shared__ int32_t sD[kDelaysInShared];  // the candidate's delay row (when it fits)
    constexpr int RPW = 2 * S / NWARP;  // image rows per warp (half DM-time, half frequency-time)
    const af_cand_t cd = cands[blockIdx.x];
    const int d = cd.dm_idx;
    __nv_bfloat16* o = out + (int64_t)blockIdx.x * S * S * 2;
    if (d < 0 || d >= ndm) {  // not a row of this plan: zero cut-outs
        for (int e = threadIdx.x; e < S * S * 2; e += T) o[e] = __float2bfloat16(0.f);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = cd.width / 2 > 1 ? cd.width / 2 : 1;
    const int64_t start = (int64_t)cd.t - 32 * (int64_t)b;
    const int span = S * b;
    const int gsz = nchan / S;
    int32_t* wp = pos[warp];
    const bool dsh = nchan <= kDelaysInShared;
    if (dsh)
        for (int c = threadIdx.x; c < nchan; c += T) sD[c] = __ldg(D + (int64_t)d * nchan + c);
    __syncthreads();
    const int32_t* Drow = dsh ? sD : D + (int64_t)d * nchan;

    // bins[k][h]: image row r = warp + NWARP*k (k < 8: DM-time row r; k >= 8:
    // frequency-time row r - 64), column 2*lane + h
    long long bins[RPW][2];
#pragma unroll
    for (int k = 0; k < RPW; k++) {
        const bool ft = k >= RPW / 2;
        const int i = warp + NWARP * (ft ? k - RPW / 2 : k);
        long long b0 = 0, b1 = 0;
        const int pr = d - 32 + i;       // plane row of a DM-time image row
        if (ft || (pr >= 0 && pr < ndm)) {
            for (int p0 = 0; p0 < span; p0 += CH) {
                const int64_t s0 = start + p0 + 4 * lane;
                bool ok[4];
#pragma unroll
                for (int q = 0; q < 4; q++) ok[q] = p0 + 4 * lane + q < span && s0 + q >= 0 && s0 + q < nout;
                int32_t a[4] = {0, 0, 0, 0};
                if (ft) {
                    uint32_t u[4] = {0u, 0u, 0u, 0u};
#pragma unroll 8
                    for (int c = i * gsz; c < (i + 1) * gsz; c++) {
                        const int64_t base = (int64_t)c * nsamp + Drow[c] + s0;  // >= 0 wherever ok[q]
#pragma unroll
                        for (int q = 0; q < 4; q++)
                            if (ok[q]) u[q] += __ldg(X + base + q);
                    }
#pragma unroll
                    for (int q = 0; q < 4; q++) a[q] = (int32_t)u[q];
                } else {
                    const int32_t* yr = plane + (int64_t)pr * nout;
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        if (ok[q]) a[q] = __ldg(yr + s0 + q);
                }
#pragma unroll
                for (int q = 0; q < 4; q++) wp[4 * lane + q] = a[q];
                __syncwarp();
                bin_chunk(wp, p0, b, lane, b0, b1);
                __syncwarp();
            }
        }
        bins[k][0] = b0;
        bins[k][1] = b1;
    }

    long long alo = LLONG_MAX, ahi = LLONG_MIN, flo = LLONG_MAX, fhi = LLONG_MIN;
#pragma unroll
    for (int k = 0; k < RPW; k++)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            if (k < RPW / 2) {
                alo = min(alo, bins[k][h]);
                ahi = max(ahi, bins[k][h]);
            } else {
                flo = min(flo, bins[k][h]);
                fhi = max(fhi, bins[k][h]);
            }
        }
    block_minmax(alo, ahi);
    block_minmax(flo, fhi);
    const float ad = (float)(ahi - alo) + 1e-6f, fd = (float)(fhi - flo) + 1e-6f;
#pragma unroll
    for (int k = 0; k < RPW; k++) {
        const bool ft = k >= RPW / 2;
        const int i = warp + NWARP * (ft ? k - RPW / 2 : k);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = i * S + 2 * lane + h;
            const float v = ft ? __fdiv_rn((float)(bins[k][h] - flo), fd) : __fdiv_rn((float)(bins[k][h] - alo), ad);
            o[2 * e + (ft ? 1 : 0)] = __float2bfloat16_rn(v);
        }
    }
}

}  // namespace

int nn_cutouts(const uint8_t* X, int64_t nsamp, int nchan, const int32_t* D, int ndm, const int32_t* plane,
               int64_t nout, const af_cand_t* cands, int n, __nv_bfloat16* out, cudaStream_t s)
{
    if (n <= 0) return AF_OK;
    k_cutout<<<n, T, 0, s>>>(X, nsamp, nchan, D, ndm, plane, nout, cands, out);
    return af_cuda_check(cudaGetLastError(), "cut-out launch");
}
