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
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "internal.h"
#include "nn.h"

namespace cg = cooperative_groups;

namespace {

constexpr int S = 64;
constexpr int kCl = 8;                 // CTAs per candidate (one thread-block cluster)
constexpr int T = 256, NWARP = T / 32; // threads per CTA; warp w of CTA r owns image rows 8 r + w of both images
constexpr int CH = 512;                // DM-time: window positions per chunk, 16 per lane
constexpr int CHF = 496;               // frequency-time: positions per chunk, 16 per lane of lanes 0..30
constexpr int kG = 6;                  // channels whose loads are issued together
constexpr int kDelaysInShared = 8192 / kCl;  // a CTA's channels whose delays are staged in shared memory

// Adds u[0..15], the column sums of window positions q0 .. q0 + 15 (q0 = the
// lane's first position), into the warp's 64 bins (bin j = positions
// [j b, (j+1) b); positions from 64 b on belong to no bin): one shared atomic
// per bin the lane's positions touch.
__device__ __forceinline__ void add_bins(const int32_t* u, int q0, int b, unsigned long long* wb)
{
    int bin = q0 / b, edge = (bin + 1) * b;
    long long acc = 0;  // added as two's complement: plane values may be negative
#pragma unroll
    for (int jj = 0; jj < 16; jj++) {
        if (q0 + jj == edge) {  // entering the next bin
            if (bin < S && acc) atomicAdd(wb + bin, (unsigned long long)acc);
            acc = 0;
            bin++;
            edge += b;
        }
        acc += u[jj];
    }
    if (bin < S && acc) atomicAdd(wb + bin, (unsigned long long)acc);
}

// Realigns a warp's 16-byte blocks: lane l holds own = the aligned block at
// aa + 16 l; its 16 bytes start m bytes in (m warp-uniform), so they are the
// bytes m .. m + 15 of own followed by lane l + 1's block (a shuffle), funnel-
// shifted.  Lane 31's result is not used.
__device__ __forceinline__ uint4 realign16(const uint4 own, int m)
{
    uint4 nx;
    nx.x = __shfl_down_sync(0xffffffffu, own.x, 1);
    nx.y = __shfl_down_sync(0xffffffffu, own.y, 1);
    nx.z = __shfl_down_sync(0xffffffffu, own.z, 1);
    nx.w = __shfl_down_sync(0xffffffffu, own.w, 1);
    const uint32_t sh = 8u * (uint32_t)(m & 3);
    switch (m >> 2) {  // warp-uniform
    case 0:
        return make_uint4(__funnelshift_r(own.x, own.y, sh), __funnelshift_r(own.y, own.z, sh),
                          __funnelshift_r(own.z, own.w, sh), __funnelshift_r(own.w, nx.x, sh));
    case 1:
        return make_uint4(__funnelshift_r(own.y, own.z, sh), __funnelshift_r(own.z, own.w, sh),
                          __funnelshift_r(own.w, nx.x, sh), __funnelshift_r(nx.x, nx.y, sh));
    case 2:
        return make_uint4(__funnelshift_r(own.z, own.w, sh), __funnelshift_r(own.w, nx.x, sh),
                          __funnelshift_r(nx.x, nx.y, sh), __funnelshift_r(nx.y, nx.z, sh));
    default:
        return make_uint4(__funnelshift_r(own.w, nx.x, sh), __funnelshift_r(nx.x, nx.y, sh),
                          __funnelshift_r(nx.y, nx.z, sh), __funnelshift_r(nx.z, nx.w, sh));
    }
}

// One cluster of kCl CTAs per candidate; CTA r computes DM-time rows and
// frequency-time rows 8 r .. 8 r + 7, warp w of it row 8 r + w of each image.
// Window positions q in [0, 64 b) are samples start + q, start = t - 32 b;
// samples outside [0, nout) count 0.  A warp walks its rows in chunks, lane l
// holding positions 16 l .. 16 l + 15 of the chunk (512 positions for the
// DM-time row, 496 for the frequency-time row, whose lane 31 only supplies
// the block after lane 30's): for the frequency-time row it adds the row's
// channels in 16-bit lanes -- one aligned 16-byte load per channel and lane,
// kG channels' loads issued together, realigned by a shuffle and funnel shifts
// and masked to the positions that count (byte loads when the input rows are
// not whole 16-byte blocks) -- then folds the 16 column sums into the warp's
// bins.  The images' minimum and maximum are reduced over the cluster through
// distributed shared memory; every CTA of a cluster takes the same path (one
// candidate), so both cluster barriers are reached by all of them.
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(T, 3)
k_cutout(const uint8_t* __restrict__ X, int64_t nsamp, int nchan, const int32_t* __restrict__ D, int ndm,
         const int32_t* __restrict__ plane, int64_t nout, const af_cand_t* __restrict__ cands, bool vec,
         __nv_bfloat16* __restrict__ out)
{
    __shared__ unsigned long long wbins[NWARP][2][S];  // per warp: bins of its DM-time and frequency-time rows
    __shared__ int32_t sD[kDelaysInShared];            // the delays of this CTA's channels (when they fit)
    __shared__ long long red[NWARP][4];                // per-warp min / max of both images
    __shared__ long long mm[4];                        // this CTA's: DM-time min, max, frequency-time min, max
    cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();
    const int cand = blockIdx.x / kCl;
    const af_cand_t cd = cands[cand];
    const int d = cd.dm_idx;
    __nv_bfloat16* o = out + (int64_t)cand * S * S * 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = NWARP * r + warp;  // image row of this warp (both images)
    if (d < 0 || d >= ndm) {  // not a row of this plan: zero cut-outs (the whole cluster returns here)
        for (int e = threadIdx.x; e < NWARP * S * 2; e += T) o[NWARP * r * S * 2 + e] = __float2bfloat16(0.f);
        return;
    }
    const int b = cd.width / 2 > 1 ? cd.width / 2 : 1;
    const int64_t start = (int64_t)cd.t - 32 * (int64_t)b;
    const int span = S * b;
    const int gsz = nchan / S;
    const int cb = NWARP * r * gsz, ce = cb + NWARP * gsz;  // this CTA's channels
    const bool dsh = ce - cb <= kDelaysInShared;
    if (dsh)
        for (int c = cb + threadIdx.x; c < ce; c += T) sD[c - cb] = __ldg(D + (int64_t)d * nchan + c);
    for (int e = lane; e < 2 * S; e += 32) (&wbins[warp][0][0])[e] = 0ull;
    __syncthreads();

    // DM-time row: plane row d - 32 + row (0 outside the plan)
    const int pr = d - 32 + row;
    if (pr >= 0 && pr < ndm) {
        const int32_t* yr = plane + (int64_t)pr * nout;
        for (int p0 = 0; p0 < span; p0 += CH) {
            const int q0 = p0 + 16 * lane;
            int32_t u[16];
#pragma unroll
            for (int jj = 0; jj < 16; jj++) {
                const int64_t sm = start + q0 + jj;
                u[jj] = q0 + jj < span && sm >= 0 && sm < nout ? __ldg(yr + sm) : 0;
            }
            add_bins(u, q0, b, wbins[warp][0]);
        }
    }
    // frequency-time row: channels row * gsz .. (row + 1) * gsz; lane 31
    // holds no positions (it supplies lane 30's next block)
    const int64_t total = (int64_t)nchan * nsamp;  // input bytes (a multiple of 16 when vec)
    for (int p0 = 0; p0 < span; p0 += CHF) {
        const int q0 = p0 + 16 * lane;
        const int64_t s0 = start + q0;  // sample of the lane's first position
        const bool mine = lane < 31;
        // bytes of the lane's positions that count: inside the window and the plane's time range
        uint32_t keep[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            uint32_t k4 = 0;
#pragma unroll
            for (int bb = 0; bb < 4; bb++) {
                const int jj = 4 * q + bb;
                if (mine && q0 + jj < span && s0 + jj >= 0 && s0 + jj < nout) k4 |= 0xFFu << (8 * bb);
            }
            keep[q] = k4;
        }
        int32_t u[16];  // column sums, at most 255 * nchan / 64
#pragma unroll
        for (int jj = 0; jj < 16; jj++) u[jj] = 0;
        for (int c0 = row * gsz; c0 < (row + 1) * gsz; c0 += 256) {  // 16-bit lanes hold 256 channels
            const int c1 = min(c0 + 256, (row + 1) * gsz);
            uint32_t E[4] = {0u, 0u, 0u, 0u}, O[4] = {0u, 0u, 0u, 0u};
            if (vec) {
                for (int c = c0; c < c1; c += kG) {
                    // the loads of kG channels first: the lane's aligned block
                    // wherever it lies inside the input (a block holding a byte
                    // that counts always does; the others are masked out)
                    uint4 own[kG];
                    int mk[kG];
#pragma unroll
                    for (int k = 0; k < kG; k++) {
                        mk[k] = 0;
                        own[k] = make_uint4(0u, 0u, 0u, 0u);
                        if (c + k < c1) {
                            const int32_t dc = dsh ? sD[c + k - cb] : __ldg(D + (int64_t)d * nchan + c + k);
                            const int64_t a = (int64_t)(c + k) * nsamp + dc + s0;
                            mk[k] = (int)(a & 15);  // the same in every lane
                            const int64_t aa = a - mk[k];
                            if (aa >= 0 && aa + 16 <= total) own[k] = __ldg(reinterpret_cast<const uint4*>(X + aa));
                        }
                    }
#pragma unroll
                    for (int k = 0; k < kG; k++)
                        if (c + k < c1) {  // warp-uniform
                            const uint4 v = realign16(own[k], mk[k]);
                            const uint32_t w[4] = {v.x & keep[0], v.y & keep[1], v.z & keep[2], v.w & keep[3]};
#pragma unroll
                            for (int q = 0; q < 4; q++) {
                                E[q] += w[q] & 0x00FF00FFu;
                                O[q] += __byte_perm(w[q], 0u, 0x4341);
                            }
                        }
                }
            } else {
                for (int c = c0; c < c1; c++) {
                    const int32_t dc = dsh ? sD[c - cb] : __ldg(D + (int64_t)d * nchan + c);
                    const int64_t a = (int64_t)c * nsamp + dc + s0;  // the lane's first byte (in the input where valid)
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        uint32_t acc = 0;
#pragma unroll
                        for (int bb = 0; bb < 4; bb++)
                            if ((keep[q] >> (8 * bb)) & 1u) acc |= (uint32_t)__ldg(X + a + 4 * q + bb) << (8 * bb);
                        E[q] += acc & 0x00FF00FFu;
                        O[q] += __byte_perm(acc, 0u, 0x4341);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                u[4 * q + 0] += (int32_t)(E[q] & 0xFFFFu);
                u[4 * q + 1] += (int32_t)(O[q] & 0xFFFFu);
                u[4 * q + 2] += (int32_t)(E[q] >> 16);
                u[4 * q + 3] += (int32_t)(O[q] >> 16);
            }
        }
        if (mine) add_bins(u, q0, b, wbins[warp][1]);
    }
    __syncwarp();
    long long bins[2][2];  // [DM-time, frequency-time][column 2 lane + h]
#pragma unroll
    for (int k = 0; k < 2; k++) {
        bins[k][0] = (long long)wbins[warp][k][2 * lane];
        bins[k][1] = (long long)wbins[warp][k][2 * lane + 1];
    }

    // min / max of both images: warp, CTA, then the cluster (distributed shared memory)
    long long v[4] = {min(bins[0][0], bins[0][1]), max(bins[0][0], bins[0][1]), min(bins[1][0], bins[1][1]),
                      max(bins[1][0], bins[1][1])};
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        v[0] = min(v[0], __shfl_xor_sync(0xffffffffu, v[0], o2));
        v[1] = max(v[1], __shfl_xor_sync(0xffffffffu, v[1], o2));
        v[2] = min(v[2], __shfl_xor_sync(0xffffffffu, v[2], o2));
        v[3] = max(v[3], __shfl_xor_sync(0xffffffffu, v[3], o2));
    }
    if (lane == 0)
        for (int i = 0; i < 4; i++) red[warp][i] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        long long m[4] = {LLONG_MAX, LLONG_MIN, LLONG_MAX, LLONG_MIN};
        for (int w = 0; w < NWARP; w++) {
            m[0] = min(m[0], red[w][0]);
            m[1] = max(m[1], red[w][1]);
            m[2] = min(m[2], red[w][2]);
            m[3] = max(m[3], red[w][3]);
        }
        for (int i = 0; i < 4; i++) mm[i] = m[i];
    }
    cluster.sync();  // every CTA's mm is written
    long long g[4] = {LLONG_MAX, LLONG_MIN, LLONG_MAX, LLONG_MIN};
    for (int q = 0; q < kCl; q++) {
        const long long* rm = cluster.map_shared_rank(mm, q);
        g[0] = min(g[0], rm[0]);
        g[1] = max(g[1], rm[1]);
        g[2] = min(g[2], rm[2]);
        g[3] = max(g[3], rm[3]);
    }
    cluster.sync();  // no CTA leaves while another may still read its mm
    const float ad = (float)(g[1] - g[0]) + 1e-6f, fd = (float)(g[3] - g[2]) + 1e-6f;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const bool ft = k == 1;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = row * S + 2 * lane + h;
            const float x = ft ? __fdiv_rn((float)(bins[k][h] - g[2]), fd) : __fdiv_rn((float)(bins[k][h] - g[0]), ad);
            o[2 * e + (ft ? 1 : 0)] = __float2bfloat16_rn(x);
        }
    }
}

}  // namespace

int nn_cutouts(const uint8_t* X, int64_t nsamp, int nchan, const int32_t* D, int ndm, const int32_t* plane,
               int64_t nout, const af_cand_t* cands, int n, __nv_bfloat16* out, cudaStream_t s)
{
    if (n <= 0) return AF_OK;
    if ((long long)n * kCl > 0x7fffffffLL) return af_set_error(AF_EINVAL, "cut-outs: too many candidates for one grid");
    // 16-byte loads: the input 16-byte aligned with rows of whole 16-byte blocks
    const bool vec = (reinterpret_cast<uintptr_t>(X) & 15) == 0 && nsamp % 16 == 0;
    k_cutout<<<(unsigned)n * kCl, T, 0, s>>>(X, nsamp, nchan, D, ndm, plane, nout, cands, vec, out);
    return af_cuda_check(cudaGetLastError(), "cut-out launch");
}
