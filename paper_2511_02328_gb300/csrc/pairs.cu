// pairs.cu -- exact brute-force dedispersion (Sec. 2.3) of single plans
// through shared channel-group rows.
//
//   Y[d][t] = sum_c X[c][t + D[d][c]]
//           = sum_q P(q, delta_q(d))[t + D[d][Gq]],
//   P(q, delta)[u]   = sum_{i<G} X[Gq+i][u + delta_i],  delta_0 = 0,
//   delta_q(d)_i     = D[d][Gq+i] - D[d][Gq],
//
// for groups of G = 2, 3 or 4 adjacent channels (a short last group has zeros
// for its missing channels).  The same integer sum, grouped: the channels of
// a group are added once per distinct tuple of relative delays (a group has a
// few dozen over the whole DM range and a few inside a block of neighbouring
// DMs), and the DM sums then run over group rows, nchan / G terms.
//
// Stage 1 (k_group_rows<G>) writes every row P(q, delta) as uint16 for one
// time block of L outputs; row g covers only the delays D[d][Gq] of the DMs
// that use it (element e is time T0 + B_g + e, B_g their smallest delay
// rounded down to 16).
//
// Stage 2 (k_pair_tile) is a tile kernel over rows: a block takes NW DM rows
// (one consumer warp each, DMs ascending) and TTE = 1016 outputs; a producer
// warp streams the block's row windows (one per block and row) through an
// NS-deep shared-memory ring, up to 32 windows of whole groups packed back to
// back per stage, one bulk async copy per window plus one for the chunk's
// consumer tables of (window, offset) per group, which the host computes once
// (tiles start at multiples of 8, so no offset depends on the tile).  Lane L
// of a consumer warp owns outputs 2 (L + 32 m) + k, m < 16, k < 2: one
// aligned 32-bit shared load brings the two 16-bit samples of a group, so the
// groups are bucketed by the parity r of the sample offset; one IADD3 adds two
// rows' words into the 16-bit lanes of the bucket's accumulator (at most
// 65535 / (255 G) rows between folds); a fold re-aligns bucket 1 by one
// sample (one lane shuffle) into the 32-bit output sums.
//
// Every wait is bounded (the tile kernel's error flag).  The host tables of
// every group size are built once per plan; a reservation picks the group size
// by a cost model and sizes the row buffer from a budget.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>
#include <array>
#include <vector>

#include "internal.h"
#include "ptx.cuh"

namespace {

constexpr int kPNW = 15;            // DM rows (consumer warps) per block
// Ring: up to kPSL row windows per stage (one per producer lane), packed back
// to back (a stage holds as many whole groups as fit its bytes); the depth is
// 2, 3 or 4 stages (AFGB_PAIR_STAGES at plan creation, default 3: on the
// 4096-channel workload with groups of 3, stage 2 took 19.8 / 19.2 / 21.5 ms).
constexpr int kPSL = 32;
constexpr int kPMG = 16;            // 2-sample groups per lane
constexpr int kPTTE = 1016;         // outputs per tile: a multiple of 8 below 64 * kPMG - 1
constexpr int kPTABW = 40;          // ints per (stage, warp) table: 2 starts, 2 counts, <= 34 offsets
constexpr uint32_t kPWait = afptx::kMbarWaitPolls;
constexpr int kET = 4096;           // stage 1: row samples per block
constexpr int kS1T = 256;
constexpr int kMaxDr = 32768;       // stage 1: largest range of one relative delay over a group's rows
constexpr int kMinTiles = 8;        // smallest useful time block, in tiles

inline int64_t r8(int64_t x) { return (x + 7) & ~(int64_t)7; }
inline int64_t r16(int64_t x) { return (x + 15) & ~(int64_t)15; }

typedef af_pair_args PairArgs;

// ------------------------------------------------------------------ stage 1
// Block = (group q of G channels, ET samples of the group's range); writes,
// for every row of the group, the part of those samples inside the row's own
// range.  pinfo[q] = {first row, rows, ub (the group's first delay rounded down
// to 16), length of the group's range}; rinfo[g] = {row start - ub (a multiple
// of 16), row length}; rdelta[g][i-1] = row g's delay of channel Gq+i relative
// to channel Gq; gdr[q][i-1] = the smallest and largest of those over the
// group's rows.  Channel Gq's window goes to W0, channel Gq+i's (shifted by
// the smallest delta, longer by the delta range + 4 bytes) to Wi: blocks whose
// windows lie inside the input rows copy them with aligned 16-byte loads (a
// window then starts off_i bytes into its buffer), edge blocks byte by byte
// with zeros outside the rows and for missing channels.  Words at any byte
// offset are read with a funnel shift (one shift per block and row).
template <int G>
__global__ void __launch_bounds__(kS1T)
k_group_rows(const uint8_t* __restrict__ X, int64_t nsamp, int nchan, const int4* __restrict__ pinfo,
             const int* __restrict__ gmax, const int2* __restrict__ gdr, const int32_t* __restrict__ rdelta,
             const int2* __restrict__ rinfo, const int64_t* __restrict__ rowoff, int64_t T0, int etiles, int wstride,
             int dshort, uint16_t* __restrict__ PS)
{
    constexpr int K = G - 1;
    extern __shared__ __align__(16) uint8_t sm[];
    const int tid = threadIdx.x;
    const int q = blockIdx.x / etiles;
    const int64_t e0 = (int64_t)(blockIdx.x % etiles) * kET;
    const int4 pi = __ldg(pinfo + q);
    // a time block dshort outputs shorter than the layout's needs every row
    // (and the group's range) dshort samples shorter (dshort a multiple of 16)
    if (e0 >= pi.w - dshort) return;
    // the rows overlapping [e0, e0 + ET): rows are ordered by start, so they are
    // those from the first starting after e0 - (longest row) to the first
    // starting at or after e0 + ET (each still checked below)
    int kbeg, kend;
    {
        const int lo_start = (int)(e0 - __ldg(gmax + q)), hi_start = (int)(e0 + kET);
        int a = 0, b = pi.y;
        while (a < b) {
            const int m = (a + b) >> 1;
            if (__ldg(rinfo + pi.x + m).x <= lo_start) a = m + 1;
            else b = m;
        }
        kbeg = a;
        b = pi.y;
        while (a < b) {
            const int m = (a + b) >> 1;
            if (__ldg(rinfo + pi.x + m).x < hi_start) a = m + 1;
            else b = m;
        }
        kend = a;
    }
    if (kbeg >= kend) return;
    const int c0 = G * q;
    const int64_t u0 = T0 + pi.z + e0;
    int dmn[K], bw[K], off[K + 1];
    bool fast = u0 >= 0 && u0 + kET + 48 <= nsamp;
#pragma unroll
    for (int i = 0; i < K; i++) {
        const int2 r = __ldg(gdr + (int64_t)q * K + i);
        dmn[i] = r.x;
        bw[i] = kET + (r.y - r.x) + 4;  // + the word the last funnel shift reads past
        fast = fast && c0 + 1 + i < nchan && u0 + r.x >= 0 && u0 + r.x + bw[i] + 48 <= nsamp;
    }
    const uint8_t* x0 = X + (int64_t)c0 * nsamp + u0;
    if (fast) {
        off[0] = (int)((uintptr_t)x0 & 15);
        const uint4* g0 = reinterpret_cast<const uint4*>(x0 - off[0]);
        const int n0 = (off[0] + kET + 4 + 15) >> 4;
        for (int k = tid; k < n0; k += kS1T) reinterpret_cast<uint4*>(sm)[k] = __ldg(g0 + k);
#pragma unroll
        for (int i = 0; i < K; i++) {
            const uint8_t* xi = X + (int64_t)(c0 + 1 + i) * nsamp + u0 + dmn[i];
            off[i + 1] = (int)((uintptr_t)xi & 15);
            const uint4* gi = reinterpret_cast<const uint4*>(xi - off[i + 1]);
            uint4* wi = reinterpret_cast<uint4*>(sm + kET + 48 + i * wstride);
            const int ni = (off[i + 1] + bw[i] + 4 + 15) >> 4;
            for (int k = tid; k < ni; k += kS1T) wi[k] = __ldg(gi + k);
        }
    } else {
        off[0] = 0;
        for (int k = tid; k < kET + 4; k += kS1T) {
            const int64_t u = u0 + k;
            sm[k] = (u >= 0 && u < nsamp) ? __ldg(x0 + k) : (uint8_t)0;
        }
#pragma unroll
        for (int i = 0; i < K; i++) {
            off[i + 1] = 0;
            const bool have = c0 + 1 + i < nchan;
            const uint8_t* xi = X + (int64_t)(have ? c0 + 1 + i : c0) * nsamp + u0 + dmn[i];
            uint8_t* wi = sm + kET + 48 + i * wstride;
            for (int k = tid; k < bw[i] + 4; k += kS1T) {
                const int64_t u = u0 + dmn[i] + k;
                wi[k] = (have && u >= 0 && u < nsamp) ? __ldg(xi + k) : (uint8_t)0;
            }
        }
    }
    __syncthreads();
    // thread tid takes the 4-sample words w = tid + 256 j (j < 4) of the block:
    // consecutive lanes read consecutive shared words (no bank conflicts) and
    // store consecutive 8-byte pieces of a row
    uint32_t alo[4], ahi[4];
    bool live[4];
    {
        const uint32_t* A32 = reinterpret_cast<const uint32_t*>(sm);
        const uint32_t sh = (uint32_t)(off[0] & 3) * 8u;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int w = tid + kS1T * j;
            live[j] = e0 + 4 * w < pi.w - dshort;
            const int p = (off[0] >> 2) + w;
            const uint32_t a = __funnelshift_r(A32[p], A32[p + 1], sh);
            alo[j] = __byte_perm(a, 0u, 0x4140);  // samples 0, 1 into 16-bit lanes
            ahi[j] = __byte_perm(a, 0u, 0x4342);  // samples 2, 3
        }
    }
    for (int k = kbeg; k < kend; k++) {
        const int2 ri = __ldg(rinfo + pi.x + k);
        uint32_t lo[4], hi[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            lo[j] = alo[j];
            hi[j] = ahi[j];
        }
#pragma unroll
        for (int i = 0; i < K; i++) {
            const uint32_t* W32 = reinterpret_cast<const uint32_t*>(sm + kET + 48 + i * wstride);
            const int pb = off[i + 1] + __ldg(rdelta + (int64_t)(pi.x + k) * K + i) - dmn[i];
            const uint32_t sh = (uint32_t)(pb & 3) * 8u;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int p = (pb >> 2) + tid + kS1T * j;
                const uint32_t b = __funnelshift_r(W32[p], W32[p + 1], sh);
                lo[j] += __byte_perm(b, 0u, 0x4140);
                hi[j] += __byte_perm(b, 0u, 0x4342);
            }
        }
        uint16_t* row = PS + __ldg(rowoff + pi.x + k);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t rel = e0 + 4 * (tid + kS1T * j) - ri.x;  // sample index within the row
            if (live[j] && rel >= 0 && rel < ri.y - dshort)
                *reinterpret_cast<uint2*>(row + rel) = make_uint2(lo[j], hi[j]);
        }
    }
}

// ------------------------------------------------------------------ stage 2
template <int NW, int NS>
struct PairTile {
    static __device__ __forceinline__ int2 load_cd(const PairArgs& a, int cbeg, int nchk, int kk)
    {
        return kk < nchk ? __ldg(a.chunks + cbeg + kk) : make_int2(0, 0);
    }

    // Chunk c (block-local kk) into stage st: its precomputed table block and
    // one window per row slot, all completing on the stage's full barrier.
    static __device__ __forceinline__ void produce(const PairArgs& a, uint8_t* smem, int* tab, uint32_t full_bar,
                                                   int c, const int2& cd, uint32_t bytes, uint32_t soff,
                                                   int64_t src, int st, int lane)
    {
        constexpr uint32_t TB = (uint32_t)(NW * kPTABW * 4);
        const uint32_t tot = __reduce_add_sync(0xffffffffu, bytes) + TB;
        __syncwarp();
        afptx::fence_proxy_async();  // the consumers' reads of this stage come before the copies
        if (lane == 0) {
            afptx::mbar_arrive_expect_tx(full_bar, tot);
            afptx::bulk_g2s(afptx::smem_addr(tab + st * NW * kPTABW), a.tabs + (int64_t)c * NW * kPTABW, TB,
                            full_bar);
        }
        __syncwarp();
        if (lane < cd.x && bytes)
            afptx::bulk_g2s(afptx::smem_addr(smem) + (uint32_t)(st * a.stage_bytes + soff), a.PS + src, bytes,
                            full_bar);
    }

    // Bucket 1 holds, in lane L group m, samples 2 (L + 32 m) + 1 and + 2: output
    // k = 0 takes its own upper half, k = 1 the lower half of the next lane's word
    // (lane 0 of group m + 1 for L = 31).
    static __device__ __forceinline__ void fold(uint32_t (&A)[2][kPMG], uint32_t (&Wd)[kPMG][2], int lane)
    {
        uint32_t carry = 0u;
#pragma unroll
        for (int m = kPMG - 1; m >= 0; m--) {
            const uint32_t a0 = A[0][m], a1 = A[1][m];
            const uint32_t lo1 = a1 & 0xFFFFu;
            uint32_t nx = __shfl_down_sync(0xffffffffu, lo1, 1);
            const uint32_t l0 = __shfl_sync(0xffffffffu, lo1, 0);
            if (lane == 31) nx = carry;
            carry = l0;
            Wd[m][0] += (a0 & 0xFFFFu) + (a1 >> 16);
            Wd[m][1] += (a0 >> 16) + nx;
            A[0][m] = 0u;
            A[1][m] = 0u;
        }
    }

    // DM block jb, outputs t0 .. t0 + TTE - 1 of the time block a.T0.
    static __device__ __forceinline__ void run(const PairArgs& a, uint8_t* smem, unsigned jb, int64_t t0)
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        int* tab = (int*)(smem + (size_t)NS * a.stage_bytes);
        uint64_t* bars = (uint64_t*)(tab + NS * NW * kPTABW);
        const uint32_t full0 = afptx::smem_addr(bars), empty0 = full0 + 8 * NS;
        const int cbeg = __ldg(a.chkoff + jb), nchk = __ldg(a.chkoff + jb + 1) - cbeg;

        if (threadIdx.x == 0) {
            for (int s = 0; s < NS; s++) {
                afptx::mbar_init(full0 + 8 * s, 1);
                afptx::mbar_init(empty0 + 8 * s, NW);
            }
            afptx::fence_mbar_init();
        }
        __syncthreads();

        if (warp == NW) {
            // ---------------- producer warp: chunk descriptors two ahead, slot records one ahead
            const int64_t dt = t0 - a.T0;
            int2 cda = load_cd(a, cbeg, nchk, 0), cdb = load_cd(a, cbeg, nchk, 1);
            int2 rcur = make_int2(0, 0), rnxt = make_int2(0, 0);
            int64_t scur = 0, snxt = 0;
            if (lane < cda.x) {
                rcur = __ldg(a.srec + cda.y + lane);
                scur = __ldg(a.soff + cda.y + lane) + dt;
            }
            int kk = 0;
            for (; kk < nchk; kk++) {
                const int st = kk % NS;
                const int2 cdc = load_cd(a, cbeg, nchk, kk + 2);
                rnxt = make_int2(0, 0);
                if (lane < cdb.x) {
                    rnxt = __ldg(a.srec + cdb.y + lane);
                    snxt = __ldg(a.soff + cdb.y + lane) + dt;
                }
                if (kk >= NS &&
                    !afptx::mbar_wait_bounded(empty0 + 8 * st, (uint32_t)(kk / NS - 1) & 1u, kPWait)) {
                    if (lane == 0) atomicExch(a.err, 1);
                    break;
                }
                produce(a, smem, tab, full0 + 8 * st, cbeg + kk, cda, (uint32_t)rcur.x, (uint32_t)rcur.y, scur, st,
                        lane);
                rcur = rnxt;
                scur = snxt;
                cda = cdb;
                cdb = cdc;
            }
            // (a drain wait that runs out raises the error flag like any other)
            for (int k2 = max(0, kk - NS); k2 < kk; k2++)
                if (!afptx::mbar_wait_bounded(full0 + 8 * (k2 % NS), (uint32_t)(k2 / NS) & 1u, kPWait) && lane == 0)
                    atomicExch(a.err, 1);
            return;
        }

        // ---------------- consumer warps: one DM row each
        const int drow = (int)jb * NW + warp;
        uint32_t A[2][kPMG], Wd[kPMG][2];
#pragma unroll
        for (int m = 0; m < kPMG; m++) {
            A[0][m] = A[1][m] = 0u;
            Wd[m][0] = Wd[m][1] = 0u;
        }
        const uint32_t lane4 = (uint32_t)lane * 4u;
        int npacc = 0;
        for (int kk = 0; kk < nchk; kk++) {
            const int st = kk % NS;
            if (!afptx::mbar_wait_bounded(full0 + 8 * st, (uint32_t)(kk / NS) & 1u, kPWait)) {
                if (lane == 0) atomicExch(a.err, 1);
                return;
            }
            const int* tb = tab + (st * NW + warp) * kPTABW;
            const int4 h = *reinterpret_cast<const int4*>(tb);  // starts 0, 1; counts 0, 1
            const int npc = h.z + h.w;
            if (npacc + npc > a.flush) {
                fold(A, Wd, lane);
                npacc = 0;
            }
            npacc += npc;
#pragma unroll
            for (int r = 0; r < 2; r++) {
                const int beg = r == 0 ? h.x : h.y;
                const int n = r == 0 ? h.z : h.w;
                const int* o = tb + 4 + beg;
                // the next two rows' offsets one iteration ahead (reads past the
                // bucket stay inside the table and are never used)
                int2 nx = *reinterpret_cast<const int2*>(o);
                int i = 0;
                for (; i + 2 <= n; i += 2) {
                    const int2 oo = nx;
                    nx = *reinterpret_cast<const int2*>(o + i + 2);
                    const uint8_t* p1 = smem + oo.x + lane4;
                    const uint8_t* p2 = smem + oo.y + lane4;
                    uint32_t w1[kPMG], w2[kPMG];
#pragma unroll
                    for (int m = 0; m < kPMG; m++) {
                        w1[m] = *reinterpret_cast<const uint32_t*>(p1 + 128 * m);
                        w2[m] = *reinterpret_cast<const uint32_t*>(p2 + 128 * m);
                    }
#pragma unroll
                    for (int m = 0; m < kPMG; m++) A[r][m] += w1[m] + w2[m];
                }
                if (i < n) {
                    const uint8_t* p1 = smem + nx.x + lane4;
#pragma unroll
                    for (int m = 0; m < kPMG; m++) A[r][m] += *reinterpret_cast<const uint32_t*>(p1 + 128 * m);
                }
            }
            __syncwarp();
            if (lane == 0) afptx::mbar_arrive(empty0 + 8 * st);
        }
        fold(A, Wd, lane);

        // ---- outputs and fused row sums
        const int orow = __ldg(a.perm + drow);
        long long ssum = 0, ssq = 0;
#pragma unroll
        for (int m = 0; m < kPMG; m++) {
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const int pos = 2 * (lane + 32 * m) + k;
                const int64_t t = t0 + pos;
                const uint32_t v = Wd[m][k];
                if (orow >= 0 && pos < kPTTE && t < a.tend) {
                    a.Y[(int64_t)orow * a.nout + t] = (int32_t)v;
                    ssum += (long long)v;
                    ssq += (long long)v * (long long)v;
                }
            }
        }
        if (a.stats) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
                ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
            }
            if (lane == 0 && orow >= 0) {
                atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[orow].sum), (unsigned long long)ssum);
                atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[orow].sumsq), (unsigned long long)ssq);
            }
        }
    }
};

// Grid = time tiles of the block x DM blocks, DM blocks fastest (a tile's rows
// stay in L2 while every DM block reads them).
template <int NW, int NS>
__global__ void __launch_bounds__((NW + 1) * 32, 1) k_pair_tile(const PairArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    PairTile<NW, NS>::run(a, smem, blockIdx.x % a.nblk, a.T0 + (int64_t)(blockIdx.x / a.nblk) * kPTTE);
}

// Persistent form over many plans' time blocks (a batch of beams): items
// (job, DM block, tile) in job order, DM blocks fastest, handed out by an
// atomic counter; every job carries its own tables and ring-stage size (the
// shared memory is sized for the largest).  The ring barriers are
// invalidated and initialised again between items.
template <int NW, int NS>
__global__ void __launch_bounds__((NW + 1) * 32, 1)
k_pair_persistent(const PairArgs* __restrict__ jobs, const long long* __restrict__ first, int njobs,
                  long long total, unsigned long long* counter)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ long long item_s;
    for (;;) {
        if (threadIdx.x == 0) item_s = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long item = item_s;
        if (item >= total) return;
        int lo = 0, hi = njobs - 1;  // the job holding the item: first[j] <= item < first[j + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (__ldg(first + mid) <= item) lo = mid;
            else hi = mid - 1;
        }
        const PairArgs& a = jobs[lo];
        const long long local = item - __ldg(first + lo);
        PairTile<NW, NS>::run(a, smem, (unsigned)(local % a.nblk), a.T0 + (local / a.nblk) * kPTTE);
        __syncthreads();  // every warp is done with the ring before its barriers are reset
        if (threadIdx.x == 0) {
            const uint32_t bar0 = afptx::smem_addr(smem + (size_t)NS * a.stage_bytes + (size_t)NS * NW * kPTABW * 4);
            for (int s = 0; s < 2 * NS; s++) afptx::mbar_inval(bar0 + 8 * s);
        }
    }
}

size_t tables_smem(int ns) { return (size_t)ns * kPNW * kPTABW * 4 + 2 * (size_t)ns * 8; }
int rows_wstride(int maxdr) { return (int)r16(kET + maxdr + 4 + 4 + 48); }
size_t rows_smem(int maxdr, int G) { return (size_t)kET + 48 + (size_t)(G - 1) * rows_wstride(maxdr); }

const void* tile_kernel(int ns)
{
    return ns == 4 ? (const void*)k_pair_tile<kPNW, 4>
         : ns == 3 ? (const void*)k_pair_tile<kPNW, 3>
                   : (const void*)k_pair_tile<kPNW, 2>;
}

size_t pair_budget()
{
    if (const char* b = getenv("AFGB_PAIR_BUDGET_MB")) return (size_t)atoll(b) << 20;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    return std::min<size_t>((size_t)48 << 30, tot / 5);
}

// Rates measured on GB300 at 2070 MHz (4096-channel workload, 1001 DMs, 3-deep
// ring): stage 2 moves shared-memory bytes (consumer loads + row-window
// copies) at about 40 / 37 / 31 TB/s for groups of 2 / 3 / 4 channels (fewer
// groups per chunk and more frequent folds as groups grow); stage 1 moves row
// bytes + input at about 6.9 / 6.5 / 5.4 TB/s of HBM; the channel tile kernel
// adds about 17.7 T samples/s.
constexpr double kTileAddps = 17.7e12;
inline double smem_rate(int G) { return G == 4 ? 31e12 : G == 3 ? 37e12 : 40e12; }
inline double row_rate(int G) { return G == 4 ? 5.2e12 : G == 3 ? 6.2e12 : 6.5e12; }

}  // namespace

int af_pair_tile_outputs() { return kPTTE; }
int af_pair_ring_depth(int ns) { return ns; }

void af_pairs_free(af_pair_tables* T)
{
    af_tile_tables_free(&T->tt);
    cudaFree(T->d_rdelta);
    cudaFree(T->d_gdr);
    cudaFree(T->d_chunks);
    cudaFree(T->d_chkoff);
    cudaFree(T->d_tabs);
    cudaFree(T->d_srec);
    for (auto& l : T->lay) {
        cudaFree(l.d_pinfo);
        cudaFree(l.d_gmax);
        cudaFree(l.d_rinfo);
        cudaFree(l.d_rowoff);
        cudaFree(l.d_soff);
    }
    if (T->ps_owned) cudaFree(T->d_ps);
    for (cudaEvent_t ev : T->tev) cudaEventDestroy(ev);
    *T = af_pair_tables();
}

// Host tables of channel groups of G (2 or 4) channels (once per plan).
// Leaves T->ok false, and returns AF_OK, when the plan is not suited: a block
// whose group needs more than a stage of rows, a delta range beyond the
// stage-1 window, more than 8 rows per group and block, or windows that fit
// no ring shape.
//
// Group q holds channels G q .. G q + G - 1 (fewer in the last group); a row
// is one tuple of delays relative to the group's first channel,
// (D[d][Gq+i] - D[d][Gq])_{i=1..G-1} (0 for a missing channel), and holds the
// sum over the group's channels at those shifts.  Row g spans the delays
// D[d][Gq] of the DMs with its tuple, from B_g (the smallest, rounded down to
// 16) over span_g samples; the group's range starts at ub_q = min_g B_g.
//
// With tiles and time blocks starting at multiples of 8, a consumer's sample
// offset inside its row window, e = D[d][Gq] - (window start & ~7), does not
// depend on the tile, so every warp's bucketed table of (slot, offset) per
// chunk is computed here once; a window starts (t0 - T0) after its position
// for the time block's first tile.
typedef std::array<int32_t, 3> Key;

static int build_groups(af_plan_t p, int G, af_pair_tables* T)
{
    af_pairs_free(T);
    const int nchan = p->nchan, ndm = p->ndm, NW = kPNW, K = G - 1;
    std::vector<int32_t> dsort, dmin;
    if (int rc = af_tile_tables_build(p->delays.data(), p->dms.data(), ndm, nchan, NW, 8, p->device, &T->tt, &dsort,
                                      &dmin))
        return rc;
    const int nblk = T->tt.nblk;
    const int ng = (nchan + G - 1) / G;
    const int32_t* D = p->delays.data();
    auto key_of = [&](const int32_t* row, int c0) {
        Key k = {0, 0, 0};
        for (int i = 1; i < G; i++)
            if (c0 + i < nchan) k[i - 1] = row[c0 + i] - row[c0];
        return k;
    };
    // rows of a group are stored in order of their start B_g (so that the rows
    // a stretch of samples overlaps are contiguous); rlook maps a tuple to its
    // row (per group, sorted by tuple)
    std::vector<int32_t> rb(ng + 1, 0), rdelta, rB, rspan, ub(ng);
    std::vector<std::pair<Key, int32_t>> rlook;
    std::vector<int2> gdr((size_t)ng * K);
    std::vector<std::pair<Key, int32_t>> v(ndm);  // (tuple, D[d][Gq])
    struct Row {
        Key key;
        int32_t B, span;
    };
    std::vector<Row> rows;
    int maxdr = 0;
    for (int q = 0; q < ng; q++) {
        const int c0 = G * q;
        for (int d = 0; d < ndm; d++) {
            const int32_t* row = D + (size_t)d * nchan;
            v[d] = std::make_pair(key_of(row, c0), row[c0]);
        }
        std::sort(v.begin(), v.end());
        rows.clear();
        for (int d = 0; d < ndm;) {
            int e = d;
            while (e < ndm && v[e].first == v[d].first) e++;
            const int32_t B = v[d].second & ~15;  // the run is sorted by delay
            rows.push_back(Row{v[d].first, B, v[e - 1].second - B});
            d = e;
        }
        std::stable_sort(rows.begin(), rows.end(), [](const Row& a, const Row& b) { return a.B < b.B; });
        const size_t n0 = rB.size();
        for (const Row& r : rows) {
            rlook.push_back(std::make_pair(r.key, (int32_t)rB.size()));
            for (int i = 0; i < K; i++) rdelta.push_back(r.key[i]);
            rB.push_back(r.B);
            rspan.push_back(r.span);
        }
        std::sort(rlook.begin() + n0, rlook.end());
        rb[q + 1] = (int32_t)rB.size();
        ub[q] = rB[n0];
        for (int i = 0; i < K; i++) {
            int32_t lo = INT32_MAX, hi = INT32_MIN;
            for (const Row& r : rows) {
                lo = std::min(lo, r.key[i]);
                hi = std::max(hi, r.key[i]);
            }
            gdr[(size_t)q * K + i] = make_int2(lo, hi);
            maxdr = std::max(maxdr, hi - lo);
        }
    }
    // window of the groups' first channels' block spread
    int spread = 0;
    for (int j = 0; j < nblk; j++)
        for (int c = 0; c < nchan; c += G) {
            int32_t hi = INT32_MIN;
            for (int w = 0; w < NW; w++) hi = std::max(hi, dsort[(size_t)(j * NW + w) * nchan + c]);
            spread = std::max(spread, hi - dmin[(size_t)j * nchan + c]);
        }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    const int64_t rwe = r8((int64_t)spread + 1031);
    if (spread >= (1 << 20) || maxdr > kMaxDr) return AF_OK;
    int NS = 3;
    if (const char* e = getenv("AFGB_PAIR_STAGES")) NS = std::min(4, std::max(2, atoi(e)));
    // one stage: up to kPSL windows back to back; the widest window must fit
    // (16 bytes stay free for the static shared memory of the persistent form)
    const int stage_bytes = (int)(((size_t)optin - tables_smem(NS) - 16) / NS) & ~15;
    if (2 * rwe > stage_bytes) return AF_OK;
    // chunks of whole groups, at most kPSL windows and stage_bytes each, per block; their tables
    struct Ent {
        int slot[kPNW];
        int e[kPNW];
    };
    std::vector<Ent> ents;
    std::vector<int2> chunks;
    std::vector<int32_t> chkoff(nblk + 1, 0), srow, scpart;
    std::vector<int2> srec;  // per slot: window bytes, offset inside its stage
    std::vector<int> tabs;
    std::vector<Key> dq(NW), S;
    std::vector<int32_t> d0(NW), sdm;
    int open_slots = 0, open_bytes = 0, first_slot = 0, kloc = 0;
    std::vector<int> sbyt, soffs;  // slot bytes and stage offsets of the open group
    auto flush = [&]() {
        if (ents.empty()) return;
        const int st = kloc % NS;
        const size_t base = tabs.size();
        tabs.resize(base + (size_t)NW * kPTABW, 0);
        for (int w = 0; w < NW; w++) {
            int* tb = tabs.data() + base + (size_t)w * kPTABW;
            int cnt[2] = {0, 0};
            for (const Ent& en : ents) cnt[en.e[w] & 1]++;
            int pos[2] = {0, (cnt[0] + 1) & ~1};  // bucket starts even: offsets load in pairs
            tb[0] = pos[0];
            tb[1] = pos[1];
            tb[2] = cnt[0];
            tb[3] = cnt[1];
            for (const Ent& en : ents) {
                const int r = en.e[w] & 1;
                tb[4 + pos[r]++] = st * stage_bytes + srec[first_slot + en.slot[w]].y + 2 * (en.e[w] - r);
            }
        }
        chunks.push_back(make_int2(open_slots, first_slot));
        ents.clear();
        open_slots = 0;
        open_bytes = 0;
        kloc++;
    };
    for (int j = 0; j < nblk; j++) {
        kloc = 0;
        for (int q = 0; q < ng; q++) {
            const int c0 = G * q;
            for (int w = 0; w < NW; w++) {
                const int32_t* row = dsort.data() + (size_t)(j * NW + w) * nchan;
                d0[w] = row[c0];
                dq[w] = key_of(row, c0);
            }
            S.assign(dq.begin(), dq.end());
            std::sort(S.begin(), S.end());
            S.erase(std::unique(S.begin(), S.end()), S.end());
            if ((int)S.size() > kPSL) return AF_OK;
            // one window per (block, row): from the smallest delay of the block's DMs on that row
            sdm.assign(S.size(), 0);
            sbyt.assign(S.size(), 0);
            int gbytes = 0;
            for (size_t k = 0; k < S.size(); k++) {
                int32_t lo = INT32_MAX, hi = INT32_MIN;
                for (int w = 0; w < NW; w++)
                    if (dq[w] == S[k]) {
                        lo = std::min(lo, d0[w]);
                        hi = std::max(hi, d0[w]);
                    }
                sdm[k] = lo;
                sbyt[k] = (int)(2 * r8((int64_t)(hi - lo) + 1031));
                gbytes += sbyt[k];
            }
            if (gbytes > stage_bytes) return AF_OK;
            if (open_slots + (int)S.size() > kPSL || open_bytes + gbytes > stage_bytes) flush();
            if (ents.empty()) first_slot = (int)srec.size();
            for (size_t k = 0; k < S.size(); k++) {
                const int g = std::lower_bound(rlook.begin() + rb[q], rlook.begin() + rb[q + 1],
                                               std::make_pair(S[k], INT32_MIN))->second;
                srec.push_back(make_int2(sbyt[k], open_bytes));
                open_bytes += sbyt[k];
                srow.push_back(g);
                scpart.push_back((sdm[k] & ~7) - rB[g]);
            }
            Ent en;
            for (int w = 0; w < NW; w++) {
                const int k = (int)(std::lower_bound(S.begin(), S.end(), dq[w]) - S.begin());
                en.slot[w] = open_slots + k;
                en.e[w] = d0[w] - (sdm[k] & ~7);
            }
            ents.push_back(en);
            open_slots += (int)S.size();
        }
        flush();
        chkoff[j + 1] = (int32_t)chunks.size();
    }
    // rows copied per group and block: beyond 8 the copies alone outweigh the
    // loads they save (the reservation weighs the rest)
    const double rows_per_group = (double)srec.size() / ((double)nblk * ng);
    if (rows_per_group > 8.0) return AF_OK;
    double copy = 0;
    for (const int2& r : srec) copy += r.x;
    T->G = G;
    T->np = ng;
    T->nrows = (int)rB.size();
    T->rwe = (int)rwe;
    T->maxdr = maxdr;
    T->rows_per_pair = rows_per_group;
    T->budget = pair_budget();
    T->shape = NS;
    T->stage_bytes = stage_bytes;
    T->copy_per_tile = copy;
    T->h_rb = rb;
    T->h_ub = ub;
    T->h_rB = rB;
    T->h_rspan = rspan;
    T->h_srow = srow;
    T->h_scpart = scpart;
    cudaError_t e;
    auto up = [&](void** d, const void* h, size_t n) {
        if ((e = cudaMalloc(d, n)) != cudaSuccess) return false;
        return (e = cudaMemcpy(*d, h, n, cudaMemcpyHostToDevice)) == cudaSuccess;
    };
    if (!up((void**)&T->d_rdelta, rdelta.data(), rdelta.size() * 4) ||
        !up((void**)&T->d_gdr, gdr.data(), gdr.size() * sizeof(int2)) ||
        !up((void**)&T->d_chunks, chunks.data(), chunks.size() * sizeof(int2)) ||
        !up((void**)&T->d_chkoff, chkoff.data(), chkoff.size() * 4) ||
        !up((void**)&T->d_tabs, tabs.data(), tabs.size() * 4) ||
        !up((void**)&T->d_srec, srec.data(), srec.size() * sizeof(int2))) {
        af_pairs_free(T);
        return af_cuda_check(e, "group tables");
    }
    for (auto& l : T->lay)
        if ((e = cudaMalloc(&l.d_pinfo, (size_t)ng * sizeof(int4))) != cudaSuccess ||
            (e = cudaMalloc(&l.d_gmax, (size_t)ng * sizeof(int))) != cudaSuccess ||
            (e = cudaMalloc(&l.d_rinfo, (size_t)T->nrows * sizeof(int2))) != cudaSuccess ||
            (e = cudaMalloc(&l.d_rowoff, (size_t)T->nrows * 8)) != cudaSuccess ||
            (e = cudaMalloc(&l.d_soff, srow.size() * 8)) != cudaSuccess) {
            af_pairs_free(T);
            return af_cuda_check(e, "group tables");
        }
    T->ok = true;
    return AF_OK;
}

// Groups of 2, 3 and 4 channels, all kept until a reservation picks one.
int af_pairs_build(af_plan_t p)
{
    if (int rc = build_groups(p, 2, &p->pairs)) return rc;
    if (p->nchan >= 8) {
        if (int rc = build_groups(p, 3, &p->alt[0])) return rc;
        if (int rc = build_groups(p, 4, &p->alt[1])) return rc;
    }
    return AF_OK;
}

// Row g's length for time blocks of L outputs: the last tile of a block
// starts at most L - TTE + span_g into the row, and its window (at most
// span_g + 1031 samples, rounded to 8) must fit: r16(L + 2 span_g + 32).
static int64_t row_len(const af_pair_tables* T, int g, int64_t L) { return r16(L + 2 * (int64_t)T->h_rspan[g] + 32); }

static int64_t rows_elems(const af_pair_tables* T, int64_t L)
{
    int64_t n = 0;
    for (int g = 0; g < T->nrows; g++) n += row_len(T, g, L);
    return n;
}

// Time block length for nout outputs within the budget (0: the rows do not fit).
static int64_t block_len(const af_pair_tables* T, int64_t nout, size_t max_bytes = SIZE_MAX)
{
    if (!T->ok || nout <= 0) return 0;
    const int64_t tiles = (nout + kPTTE - 1) / kPTTE;
    const int64_t cap = (int64_t)(std::min(T->budget, max_bytes) / 2);
    int64_t lo = kMinTiles, hi = tiles;
    if (rows_elems(T, lo * kPTTE) > cap) return 0;
    if (lo >= hi) return hi * kPTTE;
    while (lo < hi) {  // largest tile count within the budget
        const int64_t mid = (lo + hi + 1) / 2;
        if (rows_elems(T, mid * kPTTE) <= cap) lo = mid;
        else hi = mid - 1;
    }
    return lo * kPTTE;
}

int64_t af_pairs_block(af_plan_t p, int64_t nout) { return block_len(&p->pairs, nout); }

// Layout k (0: af_dedisperse, 1: af_search) of the row buffer for time
// blocks of L outputs; waits for the device first when it replaces a layout
// or the buffer (kernels in flight may read them).  Reservation calls only.
static int pairs_layout(af_plan_t p, int k, int64_t L)
{
    af_pair_tables* T = &p->pairs;
    af_pair_tables::Layout& ly = T->lay[k];
    if (ly.L == L) return AF_OK;
    const int64_t need = rows_elems(T, L);
    if (ly.L || (size_t)need * 2 > T->ps_bytes)
        if (int rc = af_cuda_check(cudaDeviceSynchronize(), "pair layout")) return rc;
    if ((size_t)need * 2 > T->ps_bytes) {
        if (!T->ps_owned) return af_set_error(AF_ENOBUFS, "pairs: the shared row buffer is too small");
        cudaFree(T->d_ps);
        T->d_ps = nullptr;
        T->ps_bytes = 0;
        if (cudaError_t e = cudaMalloc(&T->d_ps, (size_t)need * 2)) return af_cuda_check(e, "group rows");
        T->ps_bytes = (size_t)need * 2;
    }
    std::vector<int64_t> rowoff(T->nrows), soff(T->h_srow.size());
    std::vector<int4> pinfo(T->np);
    std::vector<int> gmax(T->np);
    std::vector<int2> rinfo(T->nrows);
    int64_t off = 0, maxlen = 0;
    for (int q = 0; q < T->np; q++) {
        int64_t end = 0, longest = 0;
        for (int g = T->h_rb[q]; g < T->h_rb[q + 1]; g++) {
            const int64_t len = row_len(T, g, L);
            rowoff[g] = off;
            off += len;
            rinfo[g] = make_int2(T->h_rB[g] - T->h_ub[q], (int)len);
            end = std::max(end, (int64_t)rinfo[g].x + len);
            longest = std::max(longest, len);
        }
        pinfo[q] = make_int4(T->h_rb[q], T->h_rb[q + 1] - T->h_rb[q], T->h_ub[q], (int)end);
        gmax[q] = (int)longest;
        maxlen = std::max(maxlen, end);
    }
    for (size_t i = 0; i < soff.size(); i++) soff[i] = rowoff[T->h_srow[i]] + T->h_scpart[i];
    ly.L = 0;
    cudaError_t e;
    if ((e = cudaMemcpy(ly.d_rowoff, rowoff.data(), rowoff.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(ly.d_soff, soff.data(), soff.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(ly.d_pinfo, pinfo.data(), pinfo.size() * sizeof(int4), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(ly.d_rinfo, rinfo.data(), rinfo.size() * sizeof(int2), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(ly.d_gmax, gmax.data(), gmax.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
        return af_cuda_check(e, "pair layout");
    ly.L = L;
    ly.maxlen = maxlen;
    return AF_OK;
}

// Predicted time (s) of group rows T in time blocks of L outputs on nout outputs.
static double rows_cost(af_plan_t p, const af_pair_tables* T, int64_t nout, int64_t L)
{
    const double tiles = (double)((nout + kPTTE - 1) / kPTTE), blocks = (double)((nout + L - 1) / L);
    const double s2 = (2.0 * T->tt.ndm_pad * T->np * (double)nout + tiles * T->copy_per_tile) / smem_rate(T->G);
    const double s1 = (blocks * 2.0 * (double)rows_elems(T, L) + (double)p->nchan * (double)(nout + p->dmax)) /
                      row_rate(T->G);
    return s1 + s2;
}

// Gives up a table set's row buffer and layouts (after the device is idle).
static int pairs_release(af_pair_tables* T)
{
    if (!T->d_ps && !T->lay[0].L && !T->lay[1].L) return AF_OK;
    if (int rc = af_cuda_check(cudaDeviceSynchronize(), "group rows release")) return rc;
    if (T->ps_owned) cudaFree(T->d_ps);
    T->d_ps = nullptr;
    T->ps_bytes = 0;
    T->ps_owned = true;
    T->lay[0].L = T->lay[1].L = 0;
    return AF_OK;
}

// Picks the group rows for nout outputs: of the group sizes (2 only unless
// larger groups are allowed; AFGB_PAIR_GROUP=2|3|4 restricts), the one
// predicted fastest within max_bytes of rows, if it beats the channel tile
// kernel (AFGB_DEDISP_KERNEL=pairs skips that comparison); it becomes
// p->pairs (a previously picked set gives up its buffer).  *L gets its time
// block; 0 when nothing suits.
// The candidate (0: p->pairs, 1, 2: p->alt) and time block the pick would
// take, or -1; changes nothing.
static int pairs_choose(af_plan_t p, int64_t nout, bool allow_larger, size_t max_bytes, int64_t* L)
{
    *L = 0;
    const af_pair_tables* cand[3] = {&p->pairs, &p->alt[0], &p->alt[1]};
    int best = -1;
    double best_t = 0;
    int64_t best_L = 0;
    for (int k = 0; k < 3; k++) {
        const af_pair_tables* T = cand[k];
        if (!T->ok || (T->G != 2 && !allow_larger) || (p->force_group && T->G != p->force_group)) continue;
        const int64_t Lk = block_len(T, nout, max_bytes);
        if (Lk <= 0) continue;
        const double t = rows_cost(p, T, nout, Lk);
        if (best < 0 || t < best_t) {
            best = k;
            best_t = t;
            best_L = Lk;
        }
    }
    if (best < 0) return -1;
    const bool tile = p->tile.ns1 > 0;  // else the one-thread-per-output kernel
    if (!p->force_pairs && tile && best_t >= (double)p->ndm * p->nchan * (double)nout / kTileAddps) return -1;
    *L = best_L;
    return best;
}

int af_pairs_pick(af_plan_t p, int64_t nout, bool allow_larger, size_t max_bytes, int64_t* L)
{
    const int best = pairs_choose(p, nout, allow_larger, max_bytes, L);
    if (best < 0) return AF_OK;
    if (best > 0) {
        af_pair_tables* cand[3] = {&p->pairs, &p->alt[0], &p->alt[1]};
        if (int rc = pairs_release(&p->pairs)) return rc;
        std::swap(p->pairs, *cand[best]);
    }
    return AF_OK;
}

size_t af_pairs_workspace(af_plan_t p, int64_t nout)
{
    int64_t L = 0;
    const int best = pairs_choose(p, nout, true, SIZE_MAX, &L);
    if (best < 0) return 0;
    const af_pair_tables* cand[3] = {&p->pairs, &p->alt[0], &p->alt[1]};
    return 2 * (size_t)rows_elems(cand[best], L);
}

// Reserves the picked group rows: the row buffer and the layouts of
// af_dedisperse and (with `search`) af_search.  Nothing when none suits.
int af_pairs_reserve(af_plan_t p, int64_t nout, bool search, bool allow_larger, size_t max_bytes)
{
    int64_t best_L = 0;
    if (int rc = af_pairs_pick(p, nout, allow_larger, max_bytes, &best_L)) return rc;
    if (best_L <= 0) return AF_OK;
    af_pair_tables* T = &p->pairs;
    if (best_L > T->lay[0].L)
        if (int rc = pairs_layout(p, 0, best_L)) return rc;
    if (search) {
        // af_search's growing time blocks, so that the input copy overlaps the
        // work: the layout holds the longest of them
        const std::vector<int64_t> blocks = af_search_block_tiles(nout, T->lay[0].L / kPTTE);
        const int64_t Lmax = *std::max_element(blocks.begin(), blocks.end()) * kPTTE;
        if (int rc = pairs_layout(p, 1, Lmax)) return rc;
    }
    return AF_OK;
}

std::vector<int64_t> af_search_block_tiles(int64_t nout, int64_t cap_tiles)
{
    // the dedispersion consumes input ~5 times slower than a pinned host copy
    // delivers it, and the copy starts before the first block: each block can
    // be 6 times the previous one and still find its input in place when the
    // previous one ends (on the 4096-channel workload: blocks of 6, 36 and 170
    // tiles; a median call of 25.43 ms, against 25.81 ms growing by 4 and
    // 25.90 ms growing by 8)
    const int64_t tiles = (nout + kPTTE - 1) / kPTTE;
    cap_tiles = std::max<int64_t>(1, cap_tiles);
    std::vector<int64_t> out;
    int64_t b = std::max<int64_t>(1, tiles / 32), done = 0;
    while (done < tiles) {
        const int64_t t = std::min(std::min(b, cap_tiles), tiles - done);
        out.push_back(t);
        done += t;
        b *= 6;
    }
    return out;
}

size_t af_pairs_reserved_bytes(af_plan_t p, int64_t nout)
{
    const int64_t L = af_pairs_block(p, nout);
    return L > 0 ? 2 * (size_t)rows_elems(&p->pairs, L) : 0;
}

size_t af_pairs_bytes(af_plan_t p, int64_t nout)
{
    const af_pair_tables* T = &p->pairs;
    if (!T->ok || nout <= 0) return 0;
    return 2 * (size_t)rows_elems(T, (nout + kPTTE - 1) / kPTTE * kPTTE);
}

int af_pairs_attach(af_plan_t p, uint16_t* buf, size_t bytes, int64_t nout)
{
    af_pair_tables* T = &p->pairs;
    if (!T->ok) return af_set_error(AF_EINVAL, "pairs: plan cannot use group rows");
    T->lay[0].L = T->lay[1].L = 0;  // until attached: the channel tile kernel
    const int64_t tiles = (nout + kPTTE - 1) / kPTTE;
    const int64_t cap = (int64_t)(bytes / 2);
    int64_t lo = std::min<int64_t>(kMinTiles, tiles), hi = tiles;
    if (rows_elems(T, lo * kPTTE) > cap) return af_set_error(AF_ENOBUFS, "pairs: shared row buffer too small");
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (rows_elems(T, mid * kPTTE) <= cap) lo = mid;
        else hi = mid - 1;
    }
    if (!p->force_pairs && p->tile.ns1 > 0 &&
        rows_cost(p, T, nout, lo * kPTTE) >= (double)p->ndm * p->nchan * (double)nout / kTileAddps)
        return AF_OK;  // this beam stays on the channel tile kernel
    if (int rc = af_cuda_check(cudaDeviceSynchronize(), "pairs attach")) return rc;
    if (T->ps_owned) cudaFree(T->d_ps);
    T->d_ps = buf;
    T->ps_bytes = bytes;
    T->ps_owned = false;
    return pairs_layout(p, 0, lo * kPTTE);
}

int af_launch_pairs_rows(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int layout, int64_t T0, cudaStream_t s,
                         int64_t Lb)
{
    af_pair_tables* T = &p->pairs;
    const af_pair_tables::Layout& ly = T->lay[layout];
    const int64_t L = ly.L;
    if (Lb <= 0) Lb = L;
    if (L <= 0 || L % kPTTE || T0 % kPTTE || Lb > L || Lb % kPTTE)
        return af_set_error(AF_EINVAL, "pairs: time block not laid out");
    const int dshort = (int)((L - Lb) & ~(int64_t)15);
    const size_t s1 = rows_smem(T->maxdr, T->G);
    const void* k1 = T->G == 4   ? (const void*)k_group_rows<4>
                     : T->G == 3 ? (const void*)k_group_rows<3>
                                 : (const void*)k_group_rows<2>;
    if (int rc = af_ensure_smem(k1, s1)) return rc;
    // a block dshort outputs shorter than the layout needs every group's range
    // dshort samples shorter: the grid covers only that
    const int etiles = (int)std::max<int64_t>(1, (ly.maxlen - dshort + kET - 1) / kET);
    const unsigned long long g1 = (unsigned long long)T->np * etiles;
    if (g1 > 0x7fffffffULL) return af_set_error(AF_EINVAL, "pairs: problem too large for one grid");
    if (T->G == 4)
        k_group_rows<4><<<(unsigned)g1, kS1T, s1, s>>>(d_in, nsamp, p->nchan, ly.d_pinfo, ly.d_gmax, T->d_gdr, T->d_rdelta,
                                                      ly.d_rinfo, ly.d_rowoff, T0, etiles, rows_wstride(T->maxdr),
                                                      dshort, T->d_ps);
    else if (T->G == 3)
        k_group_rows<3><<<(unsigned)g1, kS1T, s1, s>>>(d_in, nsamp, p->nchan, ly.d_pinfo, ly.d_gmax, T->d_gdr, T->d_rdelta,
                                                      ly.d_rinfo, ly.d_rowoff, T0, etiles, rows_wstride(T->maxdr),
                                                      dshort, T->d_ps);
    else
        k_group_rows<2><<<(unsigned)g1, kS1T, s1, s>>>(d_in, nsamp, p->nchan, ly.d_pinfo, ly.d_gmax, T->d_gdr, T->d_rdelta,
                                                      ly.d_rinfo, ly.d_rowoff, T0, etiles, rows_wstride(T->maxdr),
                                                      dshort, T->d_ps);
    return af_cuda_check(cudaGetLastError(), "group rows launch");
}

int af_pairs_block_args(af_plan_t p, int64_t nout, int layout, int64_t T0, int32_t* d_plane, af_rowstats_t* d_stats,
                        af_pair_args* out, long long* items, int64_t Lb)
{
    af_pair_tables* T = &p->pairs;
    const af_pair_tables::Layout& ly = T->lay[layout];
    int64_t L = ly.L;
    if (Lb <= 0) Lb = L;
    if (L <= 0 || L % kPTTE || T0 % kPTTE || T0 >= nout || Lb > L || Lb % kPTTE)
        return af_set_error(AF_EINVAL, "pairs: time block not laid out");
    L = Lb;
    af_pair_args& a = *out;
    a.PS = T->d_ps;
    a.chunks = T->d_chunks;
    a.chkoff = T->d_chkoff;
    a.tabs = T->d_tabs;
    a.srec = T->d_srec;
    a.soff = ly.d_soff;
    a.perm = T->tt.d_perm;
    a.stage_bytes = T->stage_bytes;
    a.flush = 65535 / (255 * T->G);
    a.nblk = (unsigned)T->tt.nblk;
    a.T0 = T0;
    a.tend = std::min(nout, T0 + L);
    a.nout = nout;
    a.Y = d_plane;
    a.stats = d_stats;
    a.err = p->d_err;
    *items = (long long)((std::min(L, nout - T0) + kPTTE - 1) / kPTTE) * (long long)T->tt.nblk;
    return AF_OK;
}

size_t af_pairs_stage2_smem(af_plan_t p, int ns) { return (size_t)ns * p->pairs.stage_bytes + tables_smem(ns); }

int af_launch_pairs_persistent(int ns, size_t smem, int grid, const af_pair_args* d_jobs, const long long* d_first,
                               int njobs, long long total, unsigned long long* d_counter, cudaStream_t s)
{
    const void* fn = ns == 4   ? (const void*)k_pair_persistent<kPNW, 4>
                     : ns == 3 ? (const void*)k_pair_persistent<kPNW, 3>
                               : (const void*)k_pair_persistent<kPNW, 2>;
    if (int rc = af_ensure_smem(fn, smem)) return rc;
    const dim3 blk((kPNW + 1) * 32);
    if (ns == 4)
        k_pair_persistent<kPNW, 4><<<grid, blk, smem, s>>>(d_jobs, d_first, njobs, total, d_counter);
    else if (ns == 3)
        k_pair_persistent<kPNW, 3><<<grid, blk, smem, s>>>(d_jobs, d_first, njobs, total, d_counter);
    else
        k_pair_persistent<kPNW, 2><<<grid, blk, smem, s>>>(d_jobs, d_first, njobs, total, d_counter);
    return af_cuda_check(cudaGetLastError(), "persistent pair tile launch");
}

int af_pairs_ring(af_plan_t p) { return p->pairs.shape; }

int af_launch_pairs_block(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int64_t nout, int32_t* d_plane,
                          af_rowstats_t* d_stats, cudaStream_t s, int layout, int64_t T0, cudaEvent_t* mid, int64_t Lb)
{
    af_pair_tables* T = &p->pairs;
    if (int rc = af_launch_pairs_rows(p, d_in, nsamp, layout, T0, s, Lb)) return rc;
    if (mid) AF_CUDA(cudaEventRecord(*mid, s));
    PairArgs a;
    long long items = 0;
    if (int rc = af_pairs_block_args(p, nout, layout, T0, d_plane, d_stats, &a, &items, Lb)) return rc;
    const size_t s2 = af_pairs_stage2_smem(p, T->shape);
    if (int rc = af_ensure_smem(tile_kernel(T->shape), s2)) return rc;
    if ((unsigned long long)items > 0x7fffffffULL) return af_set_error(AF_EINVAL, "pairs: problem too large for one grid");
    const dim3 grid2((unsigned)items), blk2((kPNW + 1) * 32);
    if (T->shape == 4)
        k_pair_tile<kPNW, 4><<<grid2, blk2, s2, s>>>(a);
    else if (T->shape == 3)
        k_pair_tile<kPNW, 3><<<grid2, blk2, s2, s>>>(a);
    else
        k_pair_tile<kPNW, 2><<<grid2, blk2, s2, s>>>(a);
    return af_cuda_check(cudaGetLastError(), "pair tile launch");
}

int af_launch_pairs(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int64_t nout, int32_t* d_plane,
                    af_rowstats_t* d_stats, cudaStream_t s)
{
    af_pair_tables* T = &p->pairs;
    const int64_t L = T->lay[0].L;
    if (L <= 0) return af_set_error(AF_EINVAL, "pairs: no row buffer reserved");
    if (d_stats)
        if (int rc = af_cuda_check(cudaMemsetAsync(d_stats, 0, (size_t)p->ndm * sizeof(af_rowstats_t), s),
                                   "pairs stats reset"))
            return rc;
    const int slot = T->tcalls > 0 ? T->tnext : -1;
    int b = 0;
    for (int64_t T0 = 0; T0 < nout; T0 += L, b++) {
        const bool rec = slot >= 0 && b < T->tblocks;
        cudaEvent_t* e = rec ? &T->tev[((size_t)slot * T->tblocks + b) * 3] : nullptr;
        if (rec) AF_CUDA(cudaEventRecord(e[0], s));
        if (int rc = af_launch_pairs_block(p, d_in, nsamp, nout, d_plane, d_stats, s, 0, T0, rec ? e + 1 : nullptr))
            return rc;
        if (rec) AF_CUDA(cudaEventRecord(e[2], s));
    }
    if (slot >= 0) {
        T->tnb[slot] = std::min(b, T->tblocks);
        T->trowbytes[slot] = 2 * rows_elems(T, L) * (int64_t)b;
        T->tcopybytes[slot] = (int64_t)((double)((nout + kPTTE - 1) / kPTTE) * T->copy_per_tile);
        T->tnext = (slot + 1) % T->tcalls;
    }
    return AF_OK;
}

extern "C" int af_dedisperse_timing(af_plan_t p, int ncalls)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (ncalls < 0 || ncalls > 4096) return af_set_error(AF_EINVAL, "af_dedisperse_timing: ncalls in 0..4096");
    af_pair_tables* T = &p->pairs;
    AF_CUDA(cudaDeviceSynchronize());
    for (cudaEvent_t ev : T->tev) cudaEventDestroy(ev);
    T->tev.clear();
    T->tcalls = T->tnext = 0;
    T->tblocks = 8;
    if (ncalls == 0) return AF_OK;
    T->tev.assign((size_t)ncalls * T->tblocks * 3, nullptr);
    for (cudaEvent_t& ev : T->tev)
        if (cudaError_t e = cudaEventCreate(&ev)) return af_cuda_check(e, "af_dedisperse_timing");
    T->tnb.assign(ncalls, 0);
    T->trowbytes.assign(ncalls, 0);
    T->tcopybytes.assign(ncalls, 0);
    T->tcalls = ncalls;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_dedisperse_timing");
}

extern "C" int af_dedisperse_times(af_plan_t p, int call, float* rows_ms, float* tiles_ms, int64_t* row_bytes,
                                   int64_t* copy_bytes)
try {
    if (int rc = af_check_plan(p)) return rc;
    af_pair_tables* T = &p->pairs;
    if (call < 0 || call >= T->tcalls) return af_set_error(AF_EINVAL, "af_dedisperse_times: no such call slot");
    float r = 0.f, t = 0.f;
    for (int b = 0; b < T->tnb[call]; b++) {
        cudaEvent_t* e = &T->tev[((size_t)call * T->tblocks + b) * 3];
        float x = 0.f, y = 0.f;
        AF_CUDA(cudaEventSynchronize(e[2]));
        AF_CUDA(cudaEventElapsedTime(&x, e[0], e[1]));
        AF_CUDA(cudaEventElapsedTime(&y, e[1], e[2]));
        r += x;
        t += y;
    }
    if (rows_ms) *rows_ms = r;
    if (tiles_ms) *tiles_ms = t;
    if (row_bytes) *row_bytes = T->trowbytes[call];
    if (copy_bytes) *copy_bytes = T->tcopybytes[call];
    return AF_OK;
} catch (...) {
    return af_host_exception("af_dedisperse_times");
}
