// dedisp.cu -- brute-force incoherent dedispersion (Sec. 2.3) and row sums.
//
//   Y[d][t] = sum_c X[c][t + D[d][c]],  0 <= t < nout,  exact int32.
//
// Main kernel (k_dedisp_tile): one block = NW DM rows (one per warp, DMs taken
// in ascending order so a block's delays per channel span the least) x one
// time tile of TTE outputs.  Channels stream through shared memory CC at a
// time in an NSTAGE-deep ring: for every channel one bulk async copy
// (cp.async.bulk, mbarrier completion) brings the byte window
// [t0 + Dmin_c, t0 + Dmax_c + 128*M) of that channel, 16-byte aligned.
//
// Inner loop: lane L of a warp owns outputs t0 + 4*(L + 32*m) + {0,1,2,3},
// m < M.  For channel c its DM's samples start at byte p = t0 + D[d][c]; the
// lane reads the ALIGNED 32-bit word at floor4(p) + 4*(L + 32*m) -- one
// conflict-free 128-byte wavefront per warp -- whose bytes are the samples of
// outputs shifted by r = p mod 4.  Channels are therefore bucketed by r and
// each bucket accumulates into its own set of registers; every 256 channels
// (and at the end) the sets are re-aligned with two lane shuffles and added
// into output-aligned 32-bit sums.  Bytes are widened two at a time into
// 16-bit lanes and summed exactly (at most 256 * 255 per lane between folds):
//     E += w & 0x00FF00FF            (bytes 0 and 2; one LOP3)
//     O += prmt(w, 0, 0x4341)        (bytes 1 and 3; one PRMT)
// Per word (4 sample-additions): 1 shared load, 2 ALU ops for the widening,
// 2 adds that the compiler can place on the FMA pipe.
//
// Fallback kernel (k_dedisp_simple): for plans whose per-block delay spread
// does not fit the shared-memory window (very coarse DM grids); one output
// column per thread, input read through L1.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "internal.h"
#include "ptx.cuh"

namespace {

// ------------------------------------------------------------ tile kernel
// Compile-time shape (defaults are the measured best on GB300).
#ifndef AF_TILE_M
#define AF_TILE_M 8          // 128-output groups per lane
#endif
#ifndef AF_TILE_NW
#define AF_TILE_NW 11        // consumer warps = DM rows per block
#endif
#ifndef AF_TILE_NSTAGE
#define AF_TILE_NSTAGE 4     // depth of the shared-memory ring
#endif
#ifndef AF_TILE_ADD_MODE
#define AF_TILE_ADD_MODE 0   // 0: all adds IADD3 (ALU); 1: all x*one+acc (FMA pipe);
                             // 2: bytes 0/2 by IADD3 pairs, bytes 1/3 by x*one+acc
#endif

constexpr int M = AF_TILE_M;
constexpr int NW = AF_TILE_NW;
constexpr int NT = (NW + 1) * 32;  // + one producer warp
constexpr int CC = 32;             // channels per stage (one per producer lane)
constexpr int NSTAGE = AF_TILE_NSTAGE;
constexpr int TTE = 128 * M - 4;   // outputs per tile that every bucket covers
constexpr int TABW = 48;           // ints per (stage, warp) table: 4 starts, 4 counts, 40 offsets
                                   // (at most 35 used; the slack absorbs one-pair-ahead reads)
constexpr uint32_t WAIT_LIMIT = 1u << 24;
constexpr int FLUSH_CHUNKS = 256 / CC;

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
    uint32_t one;           // 1 (opaque to the compiler: keeps the adds on the FMA pipe)
};

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Global inputs of one chunk for one producer lane (its channel): the
// block's smallest delay and the delay of every consumer warp's DM.
struct ChunkIn {
    int dmin;
    int dl[NW];
};

__device__ __forceinline__ void load_chunk(const TileArgs& a, ChunkIn& in, int kk, int jb, int lane)
{
    const int c = kk * CC + lane;
    if (kk < a.nchunks && c < a.nchan) {
        in.dmin = __ldg(a.dminblk + (int64_t)jb * a.nchan + c);
#pragma unroll
        for (int w = 0; w < NW; w++) in.dl[w] = __ldg(a.dsort + (int64_t)(jb * NW + w) * a.nchan + c);
    } else {
        in.dmin = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) in.dl[w] = 0;
    }
}

// Producer warp, chunk kk into stage st (inputs already loaded): the bucketed
// offset tables of all consumer warps, the tail bytes of windows that end in
// the last 15 bytes of the input, then the barrier's expected bytes and the
// bulk copies.
__device__ __forceinline__ void produce_chunk(const TileArgs& a, uint8_t* smem, int* tab, uint32_t full_bar,
                                              const ChunkIn& in, int kk, int st, int64_t t0, int lane)
{
    const int c = kk * CC + lane;
    const bool valid = c < a.nchan;
    int64_t start = 0;
    uint32_t bulk = 0, tail = 0;
    if (valid) {
        start = ((int64_t)c * a.nsamp + t0 + in.dmin) & ~(int64_t)15;
        const int64_t want = min((int64_t)a.rw, a.total - start);
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
            s += (cnt + 1) & ~1;   // bucket starts stay even: pairs load as 8 bytes
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
        afptx::mbar_arrive_expect_tx(full_bar, tot);   // release: tables and tails are visible
    }
    __syncwarp();
    if (valid && bulk) {
        afptx::fence_proxy_async();
        afptx::bulk_g2s(afptx::smem_addr(smem) + (uint32_t)((st * CC + lane) * a.rw), a.X + start, bulk, full_bar);
    }
}

__device__ __forceinline__ uint32_t acc_imad(uint32_t acc, uint32_t x, uint32_t one) { return x * one + acc; }

// Adds the four buckets into the output-aligned sums and clears them.  Byte k
// of bucket r in lane L, group m belongs to output 4*(L + 32*m) + k - r.  So
// output k of lane L takes byte k + r of its own word when k + r <= 3, else
// byte k + r - 4 of lane L+1's word (lane 0 of group m+1 for L = 31).
__device__ __forceinline__ void fold_buckets(uint32_t (&E)[4][M], uint32_t (&O)[4][M], uint32_t (&Wd)[M][4], int lane)
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

__global__ void __launch_bounds__(NT, 1) k_dedisp_tile(const TileArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // consecutive blocks take all DM blocks of one time tile: the input window of
    // a time tile stays resident in L2 while every DM block reads it
    const unsigned jb = blockIdx.x % a.nblk;
    const int64_t t0 = (int64_t)(blockIdx.x / a.nblk) * TTE;
    int* tab = (int*)(smem + (size_t)NSTAGE * CC * a.rw);
    uint64_t* bars = (uint64_t*)(tab + NSTAGE * NW * TABW);
    const uint32_t full0 = afptx::smem_addr(bars), empty0 = full0 + 8 * NSTAGE;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; s++) {
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
            const int st = kk % NSTAGE;
            load_chunk(a, nxt, kk + 1, (int)jb, lane);
            if (kk >= NSTAGE &&
                !afptx::mbar_wait_bounded(empty0 + 8 * st, (uint32_t)(kk / NSTAGE - 1) & 1u, WAIT_LIMIT)) {
                if (lane == 0) atomicExch(a.err, 1);
                break;
            }
            produce_chunk(a, smem, tab, full0 + 8 * st, cur, kk, st, t0, lane);
            cur = nxt;
        }
        // leave no copy in flight behind (the consumers normally wait for all of them)
        for (int k2 = max(0, kk - NSTAGE); k2 < kk; k2++)
            afptx::mbar_wait_bounded(full0 + 8 * (k2 % NSTAGE), (uint32_t)(k2 / NSTAGE) & 1u, WAIT_LIMIT);
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
    const uint32_t one = a.one;
    for (int kk = 0; kk < a.nchunks; kk++) {
        const int st = kk % NSTAGE;
        if (!afptx::mbar_wait_bounded(full0 + 8 * st, (uint32_t)(kk / NSTAGE) & 1u, WAIT_LIMIT)) {
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
            // the next pair's offsets are loaded one iteration ahead (reads past the
            // bucket stay inside the table and are never used)
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
                    const uint32_t e1 = w1[m] & 0x00FF00FFu, e2 = w2[m] & 0x00FF00FFu;
                    const uint32_t o1 = __byte_perm(w1[m], 0u, 0x4341), o2 = __byte_perm(w2[m], 0u, 0x4341);
#if AF_TILE_ADD_MODE == 0
                    E[r][m] += e1 + e2;
                    O[r][m] += o1 + o2;
#elif AF_TILE_ADD_MODE == 1
                    E[r][m] = acc_imad(acc_imad(E[r][m], e1, one), e2, one);
                    O[r][m] = acc_imad(acc_imad(O[r][m], o1, one), o2, one);
#else
                    E[r][m] += e1 + e2;
                    O[r][m] = acc_imad(acc_imad(O[r][m], o1, one), o2, one);
#endif
                }
            }
            if (i < n) {
                const uint8_t* p1 = smem + nxt.x + lane4;
#pragma unroll
                for (int m = 0; m < M; m++) {
                    const uint32_t w1 = *reinterpret_cast<const uint32_t*>(p1 + 128 * m);
                    E[r][m] = acc_imad(E[r][m], w1 & 0x00FF00FFu, one);
                    O[r][m] = acc_imad(O[r][m], __byte_perm(w1, 0u, 0x4341), one);
                }
            }
        }
        __syncwarp();
        if (lane == 0) afptx::mbar_arrive(empty0 + 8 * st);   // this warp is done with stage st
        if ((kk % FLUSH_CHUNKS) == FLUSH_CHUNKS - 1 || kk == a.nchunks - 1) fold_buckets(E, O, Wd, lane);
    }

    // ---- outputs
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

size_t tile_smem_bytes(int rw)
{
    return (size_t)NSTAGE * CC * rw + (size_t)NSTAGE * NW * TABW * sizeof(int) + 2 * NSTAGE * 8;
}

// ------------------------------------------------------------ fallback kernel
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

// Plan-time tables of the tile kernel: DMs sorted ascending (ties keep list
// order), padded to a multiple of NW by repeating the last one; the smallest
// delay of each block per channel; the window size rw.
int af_prepare_dedisp_tables(af_plan_t p)
{
    const int ndm = p->ndm, nchan = p->nchan;
    std::vector<int> order(ndm);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return p->dms[a] < p->dms[b]; });
    const int nblk = (ndm + NW - 1) / NW;
    const int ndm_pad = nblk * NW;
    std::vector<int32_t> dsort((size_t)ndm_pad * nchan), perm(ndm_pad, -1), dmin((size_t)nblk * nchan);
    for (int s = 0; s < ndm_pad; s++) {
        const int src = order[s < ndm ? s : ndm - 1];
        if (s < ndm) perm[s] = src;
        std::copy(p->delays.begin() + (size_t)src * nchan, p->delays.begin() + (size_t)(src + 1) * nchan,
                  dsort.begin() + (size_t)s * nchan);
    }
    int32_t spread = 0;
    for (int j = 0; j < nblk; j++)
        for (int c = 0; c < nchan; c++) {
            int32_t lo = INT32_MAX, hi = INT32_MIN;
            for (int w = 0; w < NW; w++) {
                const int32_t d = dsort[(size_t)(j * NW + w) * nchan + c];
                lo = std::min(lo, d);
                hi = std::max(hi, d);
            }
            dmin[(size_t)j * nchan + c] = lo;
            spread = std::max(spread, hi - lo);
        }
    // window: 15 bytes of alignment slack + spread + 128*M bytes read per warp
    const int64_t rw = ((int64_t)15 + spread + 128 * M + 15) & ~(int64_t)15;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    p->tile_ok = rw < (1 << 20) && tile_smem_bytes((int)rw) <= (size_t)optin;
    p->tile_rw = (int)std::min<int64_t>(rw, 1 << 20);
    p->dm_block = NW;
    p->n_dm_blocks = nblk;
    p->ndm_pad = ndm_pad;
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_dsort, dsort.size() * 4)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_dsort, dsort.data(), dsort.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_perm, perm.size() * 4)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_perm, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_dmin_blk, dmin.size() * 4)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_dmin_blk, dmin.data(), dmin.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_err, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(p->d_err, 0, sizeof(int))) != cudaSuccess)
        return af_cuda_check(e, "af_plan: dedispersion tables");
    if (p->tile_ok) {
        e = cudaFuncSetAttribute(k_dedisp_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes(p->tile_rw));
        if (e != cudaSuccess) return af_cuda_check(e, "af_plan: tile kernel shared memory");
    }
    return AF_OK;
}

int af_launch_dedisperse(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int64_t nout, int32_t* d_plane,
                         af_rowstats_t* d_stats, cudaStream_t s)
{
    if (p->tile_ok && !p->force_simple) {
        if (d_stats)
            if (int rc = af_cuda_check(cudaMemsetAsync(d_stats, 0, (size_t)p->ndm * sizeof(af_rowstats_t), s),
                                       "dedisperse stats reset"))
                return rc;
        TileArgs a;
        a.X = d_in;
        a.nsamp = nsamp;
        a.total = (int64_t)p->nchan * nsamp;
        a.nchan = p->nchan;
        a.nchunks = (p->nchan + CC - 1) / CC;
        a.dsort = p->d_dsort;
        a.perm = p->d_perm;
        a.dminblk = p->d_dmin_blk;
        a.nout = nout;
        a.rw = p->tile_rw;
        a.tiles = (unsigned)((nout + TTE - 1) / TTE);
        a.nblk = (unsigned)p->n_dm_blocks;
        a.Y = d_plane;
        a.stats = d_stats;
        a.err = p->d_err;
        a.one = 1u;
        const unsigned long long nb = (unsigned long long)a.tiles * a.nblk;
        if (nb > 0x7fffffffULL) return af_set_error(AF_EINVAL, "dedisperse: problem too large for one grid");
        k_dedisp_tile<<<(unsigned)nb, NT, tile_smem_bytes(a.rw), s>>>(a);
        return af_cuda_check(cudaGetLastError(), "dedisperse launch");
    }
    const unsigned tiles = (unsigned)((nout + kThreads - 1) / kThreads);
    const unsigned long long nblk = (unsigned long long)tiles * (unsigned long long)((p->ndm + kDB - 1) / kDB);
    if (nblk > 0x7fffffffULL) return af_set_error(AF_EINVAL, "dedisperse: problem too large for one grid");
    k_dedisp_simple<<<(unsigned)nblk, kThreads, 0, s>>>(d_in, nsamp, p->nchan, p->d_delays, p->ndm, nout, d_plane,
                                                        tiles);
    if (int rc = af_cuda_check(cudaGetLastError(), "dedisperse launch")) return rc;
    if (d_stats) return af_launch_rowstats(d_plane, p->ndm, nout, d_stats, s);
    return AF_OK;
}

int af_launch_rowstats(const int32_t* d_plane, int ndm, int64_t nout, af_rowstats_t* d_stats, cudaStream_t s)
{
    k_rowstats<<<ndm, kStatThreads, 0, s>>>(d_plane, nout, d_stats);
    return af_cuda_check(cudaGetLastError(), "rowstats launch");
}
