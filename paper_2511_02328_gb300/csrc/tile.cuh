// tile.cuh -- the dedispersion tile machinery (Sec. 2.3 brute-force sum),
// templated on the block shape so that the single-plan kernel, the
// persistent multi-beam kernel and the autotuner share one implementation.
//
//   Y[d][t] = sum_c X[c][t + D[d][c]],  0 <= t < nout,  exact int32.
//
// One tile = NW DM rows (one consumer warp each; DMs taken in ascending order
// so a block's delays per channel span the least) x TTE = 128*M - 4 outputs.
// A producer warp streams the channels through shared memory CC = 32 at a
// time in an NS-deep ring (full/empty mbarriers; NS = 4, or 3 / 2 when a
// coarse DM grid widens the windows): for every channel one
// bulk async copy (cp.async.bulk) brings the byte window
// [t0 + Dmin_c, t0 + Dmax_c + 128*M) of that channel, 16-byte aligned, and
// the producer writes each consumer warp's offset table for the chunk.
//
// Inner loop: lane L of a consumer warp owns outputs t0 + 4*(L + 32*m) + k,
// m < M, k < 4.  For channel c its DM's samples start at byte p = t0 + D; the
// lane reads the ALIGNED 32-bit word at floor4(p) + 4*(L + 32*m) -- one
// conflict-free 128-byte wavefront per warp -- whose bytes are the samples of
// outputs shifted by r = p mod 4.  Channels are therefore bucketed by r and
// each bucket accumulates into its own registers; every 256 channels (and at
// the end) the buckets are re-aligned with two lane shuffles and added into
// output-aligned 32-bit sums.  Bytes are widened two at a time into 16-bit
// lanes and summed exactly (at most 256 * 255 per lane between folds):
//     E += w & 0x00FF00FF            (bytes 0 and 2; one LOP3)
//     O += prmt(w, 0, 0x4341)        (bytes 1 and 3; one PRMT)
// two channels per IADD3.
//
// Subband mode (SUB = true; stage 1 of the two-stage subband dedispersion,
// Eq. stage1): the rows are coarse DMs, the channels are taken subband after
// subband (cps chunks of 32 per subband, short chunks padded), and at the end
// of every subband the warp folds and stores its partial sums
//     I(j, s, u) = sum_{c in s} X[c][u + D[j][c]]
// as one row of a scratch array.  The table delays are the coarse delays
// minus a per-(row, subband) stagger stag[j][s] = D[j][c_top(s)] - min over
// the block's rows of the same, so the delay spread inside a block is only
// the within-subband dispersion; the warp's output u is then t - stag[j][s].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "ptx.cuh"

namespace aftile {

constexpr int CC = 32;                 // channels per stage (one per producer lane)
constexpr int NSTAGE = 4;              // default depth of the shared-memory ring
constexpr int TABW = 48;               // ints per (stage, warp) table: 4 starts, 4 counts,
                                       // 40 offsets (at most 35 used; the slack absorbs
                                       // one-pair-ahead reads)
constexpr uint32_t WAIT_LIMIT = afptx::kMbarWaitPolls;
constexpr int FLUSH_CHUNKS = 256 / CC;

// One beam's dedispersion job (also the argument block of the kernels).
struct TileArgs {
    const uint8_t* X;
    int64_t nsamp;
    int64_t total;          // nchan * nsamp bytes
    int nchan;
    int nchunks;
    const int32_t* dsort;   // [ndm_pad][nchan] delays, DMs ascending
    const int32_t* perm;    // [ndm_pad] output row of each sorted DM, -1 = padding
    const int32_t* dminblk; // [nblk][nchan] smallest delay of each block per channel
    int64_t nout;
    int rw;                 // bytes per channel window (multiple of 16)
    unsigned tiles;
    unsigned nblk;
    int32_t* Y;
    af_rowstats_t* stats;   // may be NULL
    int* err;
    // subband mode only
    int cps;                // chunks per subband
    int nsub;
    const int32_t* sbfirst; // [nsub+1] first channel of each subband
    const int32_t* stag;    // [ndm_pad][nsub] stagger of each row and subband
    void* I;                // [nrows][nsub][ipitch] uint16 or uint32 partial sums
    int i16;                // I holds uint16
    int64_t ipitch;         // elements per I row
    int64_t li;             // valid outputs per I row in this launch
    int64_t tbase;          // time of tile 0 (the time block's first output)
};

__host__ __device__ constexpr int tte_of(int M) { return 128 * M - 4; }

// Window bytes for a block delay spread (15 bytes alignment slack + spread +
// 128*M bytes read per warp, rounded to 16).
__host__ __device__ inline int window_bytes(int spread, int M) { return (15 + spread + 128 * M + 15) & ~15; }

template <int NW, int NS = NSTAGE>
__host__ __device__ inline size_t smem_bytes(int rw)
{
    return (size_t)NS * CC * rw + (size_t)NS * NW * TABW * sizeof(int) + 2 * NS * 8;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <int NW, int M, bool SUB = false, int NS = NSTAGE>
struct Tile {
    static constexpr int NT = (NW + 1) * 32;  // + one producer warp
    static constexpr int TTE = tte_of(M);

    // Global inputs of one chunk for one producer lane (its channel).
    struct ChunkIn {
        int dmin;
        int dl[NW];
    };

    // Channel of producer lane `lane` in chunk kk, and whether it exists.
    static __device__ __forceinline__ int chan_of(const TileArgs& a, int kk, int lane, bool& valid)
    {
        if constexpr (SUB) {
            const int s = kk / a.cps;
            if (kk >= a.nchunks) {
                valid = false;
                return 0;
            }
            const int c = __ldg(a.sbfirst + s) + (kk - s * a.cps) * CC + lane;
            valid = c < __ldg(a.sbfirst + s + 1);
            return c;
        } else {
            const int c = kk * CC + lane;
            valid = kk < a.nchunks && c < a.nchan;
            return c;
        }
    }

    static __device__ __forceinline__ void load_chunk(const TileArgs& a, ChunkIn& in, int kk, int jb, int lane)
    {
        bool valid;
        const int c = chan_of(a, kk, lane, valid);
        if (valid) {
            in.dmin = __ldg(a.dminblk + (int64_t)jb * a.nchan + c);
#pragma unroll
            for (int w = 0; w < NW; w++) in.dl[w] = __ldg(a.dsort + (int64_t)(jb * NW + w) * a.nchan + c);
        } else {
            in.dmin = 0;
#pragma unroll
            for (int w = 0; w < NW; w++) in.dl[w] = 0;
        }
    }

    // Chunk kk into stage st: the bucketed offset tables of all consumer warps,
    // the tail bytes of windows that end in the last 15 bytes of the input, then
    // the barrier's expected bytes and the bulk copies.
    static __device__ __forceinline__ void produce_chunk(const TileArgs& a, uint8_t* smem, int* tab,
                                                         uint32_t full_bar, const ChunkIn& in, int kk, int st,
                                                         int64_t t0, int lane)
    {
        bool valid;
        const int c = chan_of(a, kk, lane, valid);
        int64_t start = 0;
        uint32_t bulk = 0, tail = 0;
        if (valid) {
            start = ((int64_t)c * a.nsamp + t0 + in.dmin) & ~(int64_t)15;
            int64_t want = min((int64_t)a.rw, a.total - start);
            if constexpr (SUB) want = max((int64_t)0, want);  // staggered tiles may start past the data
            bulk = (uint32_t)(want & ~(int64_t)15);
            tail = (uint32_t)(want - bulk);
        }
        const int64_t base = (int64_t)c * a.nsamp + t0;
#pragma unroll
        for (int w = 0; w < NW; w++) {
            const int64_t p = base + in.dl[w];
            const int r = (int)(p & 3);
            const uint32_t off = (uint32_t)((st * CC + lane) * a.rw) + (uint32_t)((p - r) - start);
            int* tb = tab + (st * NW + w) * TABW;
            int s = 0, pos = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const unsigned bal = __ballot_sync(0xffffffffu, valid && r == k);
                const int cnt = __popc(bal);
                if (r == k) pos = s + __popc(bal & lanemask_lt());
                if (lane == k) {
                    tb[k] = s;
                    tb[4 + k] = cnt;
                }
                s += (cnt + 1) & ~1;  // bucket starts stay even: pairs load as 8 bytes
            }
            if (valid) tb[8 + pos] = (int)off;
        }
        if (valid && tail) {
            uint8_t* sd = smem + (st * CC + lane) * a.rw + bulk;
            for (uint32_t i = 0; i < tail; i++) sd[i] = a.X[start + bulk + i];
        }
        const uint32_t tot = __reduce_add_sync(0xffffffffu, bulk);
        __syncwarp();
        if (lane == 0) {
            afptx::fence_proxy_async();
            afptx::mbar_arrive_expect_tx(full_bar, tot);  // release: tables and tails are visible
        }
        __syncwarp();
        if (valid && bulk) {
            afptx::fence_proxy_async();
            afptx::bulk_g2s(afptx::smem_addr(smem) + (uint32_t)((st * CC + lane) * a.rw), a.X + start, bulk,
                            full_bar);
        }
    }

    // Adds the four buckets into the output-aligned sums and clears them.  Byte
    // k of bucket r in lane L, group m belongs to output 4*(L + 32*m) + k - r.
    // So output k of lane L takes byte k + r of its own word when k + r <= 3,
    // else byte k + r - 4 of lane L+1's word (lane 0 of group m+1 for L = 31).
    static __device__ __forceinline__ void fold(uint32_t (&E)[4][M], uint32_t (&O)[4][M], uint32_t (&Wd)[M][4],
                                                int lane)
    {
        uint32_t carry[4][3];
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int j = 0; j < 3; j++) carry[r][j] = 0u;
#pragma unroll
        for (int m = M - 1; m >= 0; m--) {
            uint32_t S[4][4];
#pragma unroll
            for (int r = 0; r < 4; r++) {
                S[r][0] = E[r][m] & 0xFFFFu;
                S[r][1] = O[r][m] & 0xFFFFu;
                S[r][2] = E[r][m] >> 16;
                S[r][3] = O[r][m] >> 16;
                E[r][m] = 0u;
                O[r][m] = 0u;
            }
            uint32_t NX[4][3];
#pragma unroll
            for (int r = 1; r < 4; r++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    if (j < r) {
                        const uint32_t v = S[r][j];
                        uint32_t nx = __shfl_down_sync(0xffffffffu, v, 1);
                        const uint32_t l0 = __shfl_sync(0xffffffffu, v, 0);
                        if (lane == 31) nx = carry[r][j];
                        NX[r][j] = nx;
                        carry[r][j] = l0;
                    }
                }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                uint32_t v = 0;
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    if (k + r <= 3)
                        v += S[r][k + r];
                    else
                        v += NX[r][k + r - 4];
                }
                Wd[m][k] += v;
            }
        }
    }

    // Subband mode: writes this warp's sums of subband s as I(row, s, u) with
    // u = t0 - tbase + pos - stag[drow][s], for 0 <= u < li, and clears them.
    static __device__ __forceinline__ void store_subband(const TileArgs& a, int drow, int s, int64_t t0,
                                                         uint32_t (&Wd)[M][4], int lane)
    {
        const int orow = __ldg(a.perm + drow);
        if (orow >= 0) {
            const int64_t ub = t0 - a.tbase - (int64_t)__ldg(a.stag + (int64_t)drow * a.nsub + s);
            const int64_t rowoff = ((int64_t)orow * a.nsub + s) * a.ipitch;
#pragma unroll
            for (int m = 0; m < M; m++) {
                const int pos0 = 4 * (lane + 32 * m);
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int pos = pos0 + k;
                    const int64_t u = ub + pos;
                    if (pos < TTE && u >= 0 && u < a.li) {
                        if (a.i16)
                            reinterpret_cast<uint16_t*>(a.I)[rowoff + u] = (uint16_t)Wd[m][k];
                        else
                            reinterpret_cast<uint32_t*>(a.I)[rowoff + u] = Wd[m][k];
                    }
                }
            }
        }
#pragma unroll
        for (int m = 0; m < M; m++)
#pragma unroll
            for (int k = 0; k < 4; k++) Wd[m][k] = 0u;
    }

    // The whole block computes tile (jb, t0) of job a.  Every thread returns.
    static __device__ __forceinline__ void run(const TileArgs& a, unsigned jb, int64_t t0, uint8_t* smem)
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        int* tab = (int*)(smem + (size_t)NS * CC * a.rw);
        uint64_t* bars = (uint64_t*)(tab + NS * NW * TABW);
        const uint32_t full0 = afptx::smem_addr(bars), empty0 = full0 + 8 * NS;

        if (threadIdx.x == 0) {
            for (int s = 0; s < NS; s++) {
                afptx::mbar_init(full0 + 8 * s, 1);
                afptx::mbar_init(empty0 + 8 * s, NW);
            }
            afptx::fence_mbar_init();
        }
        __syncthreads();

        if (warp == NW) {
            // ---------------- producer warp
            // the global loads of chunk kk+1 are in flight while chunk kk is produced
            ChunkIn cur, nxt;
            load_chunk(a, cur, 0, (int)jb, lane);
            int kk = 0;
            for (; kk < a.nchunks; kk++) {
                const int st = kk % NS;
                load_chunk(a, nxt, kk + 1, (int)jb, lane);
                if (kk >= NS &&
                    !afptx::mbar_wait_bounded(empty0 + 8 * st, (uint32_t)(kk / NS - 1) & 1u, WAIT_LIMIT)) {
                    if (lane == 0) atomicExch(a.err, 1);
                    break;
                }
                produce_chunk(a, smem, tab, full0 + 8 * st, cur, kk, st, t0, lane);
                cur = nxt;
            }
            // leave no copy in flight behind (the consumers normally wait for all of them)
            // (a drain wait that runs out raises the error flag like any other)
            for (int k2 = max(0, kk - NS); k2 < kk; k2++)
                if (!afptx::mbar_wait_bounded(full0 + 8 * (k2 % NS), (uint32_t)(k2 / NS) & 1u, WAIT_LIMIT) && lane == 0)
                    atomicExch(a.err, 1);
            return;
        }

        // ---------------- consumer warps: one DM row each
        const int drow = (int)jb * NW + warp;
        uint32_t E[4][M], O[4][M], Wd[M][4];
#pragma unroll
        for (int m = 0; m < M; m++) {
#pragma unroll
            for (int r = 0; r < 4; r++) E[r][m] = O[r][m] = 0u;
#pragma unroll
            for (int k = 0; k < 4; k++) Wd[m][k] = 0u;
        }
        const uint32_t lane4 = (uint32_t)lane * 4u;
        int sb = 0, sq = 0;  // subband mode: current subband and chunk within it
        for (int kk = 0; kk < a.nchunks; kk++) {
            const int st = kk % NS;
            if (!afptx::mbar_wait_bounded(full0 + 8 * st, (uint32_t)(kk / NS) & 1u, WAIT_LIMIT)) {
                if (lane == 0) atomicExch(a.err, 1);
                return;
            }
            const int* tb = tab + (st * NW + warp) * TABW;
            const int4 begs = *reinterpret_cast<const int4*>(tb);
            const int4 cnts = *reinterpret_cast<const int4*>(tb + 4);
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int beg = r == 0 ? begs.x : r == 1 ? begs.y : r == 2 ? begs.z : begs.w;
                const int n = r == 0 ? cnts.x : r == 1 ? cnts.y : r == 2 ? cnts.z : cnts.w;
                const int* o = tb + 8 + beg;
                // the next pair's offsets are loaded one iteration ahead (reads past
                // the bucket stay inside the table and are never used)
                int2 nxt = *reinterpret_cast<const int2*>(o);
                int i = 0;
                for (; i + 2 <= n; i += 2) {
                    const int2 oo = nxt;
                    nxt = *reinterpret_cast<const int2*>(o + i + 2);
                    const uint8_t* p1 = smem + oo.x + lane4;
                    const uint8_t* p2 = smem + oo.y + lane4;
                    uint32_t w1[M], w2[M];
#pragma unroll
                    for (int m = 0; m < M; m++) {
                        w1[m] = *reinterpret_cast<const uint32_t*>(p1 + 128 * m);
                        w2[m] = *reinterpret_cast<const uint32_t*>(p2 + 128 * m);
                    }
#pragma unroll
                    for (int m = 0; m < M; m++) {
                        E[r][m] += (w1[m] & 0x00FF00FFu) + (w2[m] & 0x00FF00FFu);
                        O[r][m] += __byte_perm(w1[m], 0u, 0x4341) + __byte_perm(w2[m], 0u, 0x4341);
                    }
                }
                if (i < n) {
                    const uint8_t* p1 = smem + nxt.x + lane4;
#pragma unroll
                    for (int m = 0; m < M; m++) {
                        const uint32_t w1 = *reinterpret_cast<const uint32_t*>(p1 + 128 * m);
                        E[r][m] += w1 & 0x00FF00FFu;
                        O[r][m] += __byte_perm(w1, 0u, 0x4341);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) afptx::mbar_arrive(empty0 + 8 * st);  // this warp is done with stage st
            if constexpr (SUB) {
                const bool last = sq == a.cps - 1;
                if ((sq % FLUSH_CHUNKS) == FLUSH_CHUNKS - 1 || last) fold(E, O, Wd, lane);
                if (last) {
                    store_subband(a, drow, sb, t0, Wd, lane);
                    sq = 0;
                    sb++;
                } else {
                    sq++;
                }
            } else {
                if ((kk % FLUSH_CHUNKS) == FLUSH_CHUNKS - 1 || kk == a.nchunks - 1) fold(E, O, Wd, lane);
            }
        }
        if constexpr (SUB) return;

        // ---- outputs and fused row sums
        const int orow = a.perm[drow];
        long long ssum = 0, ssq = 0;
#pragma unroll
        for (int m = 0; m < M; m++) {
            const int pos0 = 4 * (lane + 32 * m);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int pos = pos0 + k;
                const int64_t t = t0 + pos;
                const uint32_t v = Wd[m][k];
                if (orow >= 0 && pos < TTE && t < a.nout) {
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

// Grid = tiles x DM blocks of one job, tile 0 starting at output a.tbase.
// Consecutive blocks take all DM blocks of one time tile, so the input window
// of a time tile stays resident in L2 while every DM block reads it.
template <int NW, int M, int NS = NSTAGE>
__global__ void __launch_bounds__((NW + 1) * 32, 1) k_tile(const TileArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const unsigned jb = blockIdx.x % a.nblk;
    const int64_t t0 = a.tbase + (int64_t)(blockIdx.x / a.nblk) * Tile<NW, M, false, NS>::TTE;
    Tile<NW, M, false, NS>::run(a, jb, t0, smem);
}

// Stage 1 of the subband dedispersion: grid = tiles x row blocks, tile 0
// starting at a.tbase.
template <int NW, int M>
__global__ void __launch_bounds__((NW + 1) * 32, 1) k_tile_sb(const TileArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const unsigned jb = blockIdx.x % a.nblk;
    const int64_t t0 = a.tbase + (int64_t)(blockIdx.x / a.nblk) * Tile<NW, M, true>::TTE;
    Tile<NW, M, true>::run(a, jb, t0, smem);
}

// Persistent multi-job kernel: each block takes work items (job, DM block,
// time tile) from a global counter until all `total` items are done.  Item i
// belongs to the job b with first[b] <= i < first[b+1]; within a job the
// order is DM block fastest, then time tile.  The job is copied to shared
// memory; the ring's barriers are invalidated and re-initialised per item.
template <int NW, int M>
__global__ void __launch_bounds__((NW + 1) * 32, 1)
k_tile_persistent(const TileArgs* __restrict__ jobs, const long long* __restrict__ first, int njobs,
                  long long total, unsigned long long* counter)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ TileArgs s_job;
    __shared__ long long s_item;
    __shared__ int s_b;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long it = (long long)atomicAdd(counter, 1ull);
            s_item = it;
            int b = 0;
            if (it < total)
                while (b + 1 < njobs && first[b + 1] <= it) b++;
            s_b = b;
            if (it < total) s_job = jobs[b];
        }
        __syncthreads();
        const long long it = s_item;
        if (it >= total) break;
        const long long local = it - first[s_b];
        const unsigned jb = (unsigned)(local % s_job.nblk);
        const int64_t t0 = (int64_t)(local / s_job.nblk) * Tile<NW, M>::TTE;
        Tile<NW, M>::run(s_job, jb, t0, smem);
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint32_t full0 = afptx::smem_addr(smem + (size_t)NSTAGE * CC * s_job.rw +
                                                    (size_t)NSTAGE * NW * TABW * sizeof(int));
            for (int s = 0; s < 2 * NSTAGE; s++) afptx::mbar_inval(full0 + 8 * s);
        }
        __syncthreads();
    }
}

}  // namespace aftile
