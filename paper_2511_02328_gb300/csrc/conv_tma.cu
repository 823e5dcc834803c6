// conv_tma.cu -- the classifier's 3x3 convolutions (pad 1) on the tcgen05
// tensor cores, every operand tile staged in shared memory by bulk async
// copies (the TMA unit).  The classifier replaces the paper's YOLO detector
// (Sec. 2.5).
//
// Activations and activation gradients of this path are channel-blocked:
// [n][C/8][H][W][8] bf16.  The eight channels of a pixel are 16 contiguous
// bytes and eight consecutive pixels of one channel block 128 contiguous
// bytes -- one core matrix of the tensor cores' no-swizzle layout, K-major
// where the channels are the contraction (forward, data gradient), MN-major
// where the pixels are (weight gradient).
//
// A tile is R = 128 / W whole rows y0 .. y0 + R - 1 of one image (128 output
// pixels).  A stage holds three copies of rows y0 - 1 .. y0 + R of every
// channel block, copy dx shifted by dx - 1 columns (pixel (r, x) of copy dx =
// X[y0 - 1 + r][x + dx - 1]).  Each copy of a block is one contiguous run of
// the image's rows, so one bulk copy; the shift wraps a row's first (last)
// pixel to the previous (next) row's end, and once the copies have landed a
// fix warp zeroes those pixels and the rows outside the image: the
// convolution's zero padding.  Tap (dy, dx) of the filter is then copy dx
// from its row dy on, a descriptor start address; no im2col gather is made:
//
//   forward  Z[p][o]     = sum_{t,i} X[p + t][i] W[o][t][i]   A = X copies (K-major), B = W
//   dgrad    dX[p][i]    = sum_{t,o} dZ[p - t][o] W[o][t][i]  the same form on dZ, taps flipped,
//                                                            W transposed
//   wgrad    dW[o][t][i] = sum_p dZ[p][o] X[p + t][i]         A = dZ^T, B = X copies (MN-major);
//                                                            layer 1: A = X copies, B = dZ^T
//
// The first layer's input is column-expanded in shared memory: its raw
// two-channel rows are copied and the fix warp writes one block of eight
// channels holding the two channels of columns x - 1, x, x + 1 (and two
// zeros), so one plane serves every tap, a K step of 16 takes two rows dy, and
// the weight gradient takes the three rows dy along N.
//
// One warp-specialised kernel serves all three: warp 0 issues a tile's bulk
// copies (one per lane) into an NS-deep ring; warp 6 fixes a stage's padding
// once its copies have landed and releases it; warp 1 (one elected thread)
// issues the tile's MMAs into one of NACC tensor-memory accumulators and
// commits them; warps 2-5 read the accumulator back (tcgen05.ld, warp w reads
// lanes 32 (w % 4) ..) for the epilogue (in the first layer's weight
// gradient, whose accumulator is read once at the end, they first build each
// stage's output gradient from the pooled one: the pooling's backward pass).
// Each role waits on one barrier, so the roles overlap across tiles.  Every wait is bounded in wall time; a
// wait that runs out raises the caller's error flag and the block leaves.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "internal.h"
#include "nn.h"
#include "ptx.cuh"
#include "umma.cuh"

namespace {

constexpr int kThreads = 224;  // copy warp, MMA warp, four epilogue warps, fix warp
constexpr int kFixWarp = 6;
constexpr uint32_t kBackoffNs = 64;  // the copy, fix and MMA warps' polls leave issue slots to the epilogue

constexpr uint32_t align1k(uint32_t b) { return (b + 1023u) / 1024u * 1024u; }
constexpr int clampi(int v, int lo, int hi) { return v < lo ? lo : v > hi ? hi : v; }
constexpr int pow2_cols(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : n <= 256 ? 256 : 512; }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// The epilogue warps' own barrier (id 1, 128 threads).
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Barrier of the epilogue warps that also ORs a flag over them: every warp
// leaves with the same answer.
__device__ __forceinline__ bool epi_sync_any(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

// Geometry of a tile of W columns over CB channel blocks: R rows of outputs,
// a copy (one column shift) holds R + 2 rows of every block.
template <int CB, int W>
struct Geo {
    static_assert(W == 16 || W == 32 || W == 64, "tile widths");
    static constexpr int R = 128 / W;
    static constexpr uint32_t PLANE = (uint32_t)(R + 2) * W * 16;  // one channel block of a copy
    static constexpr uint32_t COPY = align1k(PLANE * CB);          // a copy, 1024-byte aligned
};

// The three shifted copies of a tile (image img, rows y0 - 1 .. y0 + R) of a
// channel-blocked tensor `in` with CB blocks of H x W pixels.  Copy c (< 3 CB)
// is block c % CB of copy dx = c / CB: the image's rows among y0 - 1 ..
// y0 + R, one run; copy 0 lands one pixel later than it starts in memory,
// copy 2 one pixel earlier.  Planes (one block of one copy) sit copy-major
// (dx * COPY + cb * PLANE) or, BM, block-major ((3 cb + dx) * PLANE).  With
// NSH = 1 (the first layer) `in` is the raw input [n][H][W][2]: its rows are
// copied after the plane and fixup() expands them into a column-expanded
// plane, whose pixels carry their own column neighbours.
template <int CB, int W, bool BM = false, int NSH = 3>
struct Halo {
    using G = Geo<CB, W>;
    static_assert(NSH == 1 || NSH == 3, "copies");
    static_assert(NSH == 3 || CB == 1, "the column-expanded form has one block");
    static constexpr int R = G::R, NCOPY = NSH * CB;
    // NSH = 1: the raw two-channel rows (4 bytes a pixel) land after the plane
    // and the fix warp expands them into it
    static constexpr uint32_t RAW = (uint32_t)(R + 2) * W * 4;
    static constexpr uint32_t BYTES = NSH == 1 ? align1k(G::PLANE + RAW) : BM ? align1k(3 * CB * G::PLANE) : 3 * G::COPY;
    __host__ __device__ static constexpr uint32_t plane(int dx, int cb)
    {
        return NSH == 1 ? (uint32_t)cb * G::PLANE
               : BM     ? (uint32_t)(3 * cb + dx) * G::PLANE
                        : (uint32_t)dx * G::COPY + (uint32_t)cb * G::PLANE;
    }
    // the image's rows ylo .. ylo + nrows - 1 land at stage row rlo
    __device__ static void rows(int y0, int H, int& ylo, int& nrows, int& rlo)
    {
        ylo = y0 > 0 ? y0 - 1 : 0;
        const int yhi = y0 + R < H ? y0 + R : H - 1;
        nrows = yhi - ylo + 1;
        rlo = ylo - (y0 - 1);
    }
    __device__ static uint32_t tx(int y0, int H)
    {
        int ylo, nrows, rlo;
        rows(y0, H, ylo, nrows, rlo);
        return NSH == 1 ? (uint32_t)nrows * W * 4 : (uint32_t)CB * (3u * (uint32_t)nrows * W * 16 - 32u);
    }
    __device__ static void copy(int c, uint32_t st, const __nv_bfloat16* in, int img, int y0, int H, uint32_t bar)
    {
        int ylo, nrows, rlo;
        rows(y0, H, ylo, nrows, rlo);
        if constexpr (NSH == 1) {  // in: the raw input [n][H][W][2]
            const uint8_t* src = reinterpret_cast<const uint8_t*>(in) + ((int64_t)img * H + ylo) * W * 4;
            afptx::bulk_g2s(st + G::PLANE + (uint32_t)rlo * W * 4, src, (uint32_t)nrows * W * 4, bar);
        } else {
            const int dx = c / CB, cb = c - dx * CB;
            const uint8_t* src = reinterpret_cast<const uint8_t*>(in) + (((int64_t)img * CB + cb) * H + ylo) * W * 16;
            const uint32_t dst = st + plane(dx, cb) + (uint32_t)rlo * W * 16;
            const uint32_t len = (uint32_t)nrows * W * 16;
            if (dx == 1) afptx::bulk_g2s(dst, src, len, bar);
            else if (dx == 0) afptx::bulk_g2s(dst + 16, src, len - 16, bar);
            else afptx::bulk_g2s(dst, src + 16, len - 16, bar);
        }
    }
    // After the copies landed: zero the wrapped pixels (column 0 of copy 0,
    // column W - 1 of copy 2, every row and block) and the rows outside the
    // image, then make the writes visible to the tensor cores.
    __device__ static void fixup(uint8_t* st, int y0, int H, int lane)
    {
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        if constexpr (NSH == 1) {
            // the column-expanded plane: pixel (r, x) = the two channels of
            // columns x - 1, x, x + 1 of raw row r (zeros outside the image), two zeros
            const uint32_t* raw = reinterpret_cast<const uint32_t*>(st + G::PLANE);
            for (int e = lane; e < (R + 2) * W; e += 32) {
                const int r = e / W, x = e - r * W, y = y0 - 1 + r;
                uint4 v = z;
                if (y >= 0 && y < H) {
                    const uint32_t* row = raw + r * W;
                    v = make_uint4(x > 0 ? row[x - 1] : 0u, row[x], x < W - 1 ? row[x + 1] : 0u, 0u);
                }
                *reinterpret_cast<uint4*>(st + e * 16) = v;
            }
        } else {
            for (int e = lane; e < 2 * CB * (R + 2); e += 32) {
                const int k = e / (CB * (R + 2)), rem = e - k * CB * (R + 2), cb = rem / (R + 2), r = rem - cb * (R + 2);
                *reinterpret_cast<uint4*>(st + plane(2 * k, cb) + (r * W + (k ? W - 1 : 0)) * 16) = z;
            }
            if (y0 == 0 || y0 + R == H) {
                const int r = y0 == 0 ? 0 : R + 1;  // R < H: a tile has one edge at most
                for (int e = lane; e < 3 * CB * W; e += 32) {
                    const int c = e / W, x = e - c * W, dx = c / CB, cb = c - dx * CB;
                    *reinterpret_cast<uint4*>(st + plane(dx, cb) + (r * W + x) * 16) = z;
                }
            }
        }
        afptx::fence_proxy_async();
    }
};

// ------------------------------------------------------------ the pipeline
// Barriers: full[s] (the bulk copies' transaction bytes), ready[s] (the fix
// warp fixed the stage), empty[s] (MMA commit), tfull[b] (MMA
// commit: accumulator b holds a finished tile), tempty[b] (128 epilogue
// arrivals: accumulator b was read).  Op provides NS, NACC, NCOL, PER_TILE (an
// epilogue per tile, else one at the end over the block's tiles), RB
// (resident bytes, a multiple of 1024), SSTAGE, SLACK (bytes after the ring
// that MMAs may read), NCOPY, ntiles(), tx(), copy(), fixup(), resident(),
// mma(), epilogue(), final().
template <class Op>
__global__ void __launch_bounds__(kThreads) k_tconv(const typename Op::Args args)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[3 * Op::NS + 2 * Op::NACC];
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    __shared__ __align__(16) float xv[32 * 16];  // pool exchange between epilogue warps
    __shared__ uint32_t xq[64];
    constexpr int NS = Op::NS, NACC = Op::NACC;
    constexpr uint32_t TCOLS = pow2_cols(NACC * Op::NCOL);
    static_assert(Op::NCOPY <= 32, "one bulk copy per producer lane");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const Op op(args);
    const int ntiles = op.ntiles();
    const int mytiles = ntiles > (int)blockIdx.x ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    const uint32_t raw = afptx::smem_addr(smem_raw), base = (raw + 1023u) & ~1023u;
    uint8_t* sm = smem_raw + (base - raw);
    const uint32_t ring = base + Op::RB;
    const uint32_t full0 = afptx::smem_addr(bars), ready0 = full0 + 8 * NS, empty0 = ready0 + 8 * NS,
                   tfull0 = empty0 + 8 * NS, tempty0 = tfull0 + 8 * NACC;
    volatile int* abort = &abort_flag;
    auto tile_of = [&](int g) { return (int)blockIdx.x + g * (int)gridDim.x; };

    if (tid == 0) {
        for (int s = 0; s < NS; s++) {
            afptx::mbar_init(full0 + 8 * s, Op::FULL_ARRIVALS);
            afptx::mbar_init(ready0 + 8 * s, 1);
            afptx::mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < NACC; b++) {
            afptx::mbar_init(tfull0 + 8 * b, 1);
            afptx::mbar_init(tempty0 + 8 * b, 128);
        }
        abort_flag = 0;
        afptx::fence_mbar_init();
    }
    if (warp == 1) {
        afumma::tmem_alloc(afptx::smem_addr(&tslot), TCOLS);
        afumma::tmem_relinquish();
    }
    op.resident(sm, tid);  // resident weights (generic stores)
    if constexpr (Op::SLACK > 0)
        for (uint32_t i = tid; i < Op::SLACK / 16; i += kThreads)
            reinterpret_cast<uint4*>(sm + Op::RB + NS * Op::SSTAGE)[i] = make_uint4(0u, 0u, 0u, 0u);
    afptx::fence_proxy_async();  // ... visible to the tensor cores
    afumma::fence_before_sync();
    __syncthreads();
    afumma::fence_after_sync();
    const uint32_t tmem = tslot;

    if (warp == 0) {
        // ---------------- copies: tile g into stage g % NS once the MMAs of tile g - NS are done
        int g = 0;
        for (; g < mytiles; g++) {
            const int s = g % NS;
            if (g >= NS && !__all_sync(0xffffffffu, afumma::wait_or_abort(empty0 + 8 * s, (uint32_t)(g / NS - 1) & 1u,
                                                                           abort, kBackoffNs)))
                break;
            if (lane == 0) afptx::mbar_arrive_expect_tx(full0 + 8 * s, op.tx(tile_of(g)));
            __syncwarp();
            if (lane < Op::NCOPY) op.copy(lane, ring + (uint32_t)s * Op::SSTAGE, tile_of(g), full0 + 8 * s);
        }
        // the last copies land before the block's shared memory goes away (a
        // bounded wait that an abort does not cut short)
        if (lane == 0)
            for (int h = g - NS < 0 ? 0 : g - NS; h < g; h++) {
                const uint64_t t0 = afumma::globaltimer_ns();
                while (!afumma::mbar_test_wait(full0 + 8 * (h % NS), (uint32_t)(h / NS) & 1u) &&
                       afumma::globaltimer_ns() - t0 < afumma::kWaitNs) {
                }
            }
    } else if (warp == kFixWarp) {
        // ---------------- fixes: tile g's padding once its copies have landed, then the stage is ready
        int g = 0;
        for (; g < mytiles; g++) {
            const int s = g % NS;
            if (!__all_sync(0xffffffffu, afumma::wait_or_abort(full0 + 8 * s, (uint32_t)(g / NS) & 1u, abort, kBackoffNs)))
                break;
            op.fixup(sm + Op::RB + (size_t)s * Op::SSTAGE, tile_of(g), lane);
            __syncwarp();
            if (lane == 0) afptx::mbar_arrive(ready0 + 8 * s);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        int g = 0;
        for (; g < mytiles; g++) {
            const int s = g % NS, b = g % NACC;
            bool ok = true;
            if (Op::PER_TILE && g >= NACC)  // the epilogue has read this accumulator's previous tile
                ok = afumma::wait_or_abort(tempty0 + 8 * b, (uint32_t)(g / NACC - 1) & 1u, abort, kBackoffNs);
            ok = ok && afumma::wait_or_abort(ready0 + 8 * s, (uint32_t)(g / NS) & 1u, abort, kBackoffNs);
            if (!__all_sync(0xffffffffu, ok)) break;
            afumma::fence_after_sync();
            if (lane == 0) {
                op.mma(ring + (uint32_t)s * Op::SSTAGE, base, tmem + (uint32_t)(Op::PER_TILE ? b * Op::NCOL : 0), g);
                afumma::commit(empty0 + 8 * s);
                if (Op::PER_TILE) afumma::commit(tfull0 + 8 * b);
                else if (g == mytiles - 1) afumma::commit(tfull0);
            }
            __syncwarp();
        }
        // every MMA reading the ring has completed before the block leaves
        for (int h = g - NS < 0 ? 0 : g - NS; h < g && !*abort; h++)
            afumma::wait_or_abort(empty0 + 8 * (h % NS), (uint32_t)(h / NS) & 1u, abort);
    } else {
        // ---------------- epilogue (warps 2-5)
        const int quarter = warp & 3;
        if (Op::PER_TILE) {
            for (int i = 0; i < mytiles; i++) {
                const int b = i % NACC;
                const bool ok = afumma::wait_or_abort(tfull0 + 8 * b, (uint32_t)(i / NACC) & 1u, abort);
                if (epi_sync_any(!ok || *abort)) break;  // all four warps leave together
                afumma::fence_after_sync();
                op.epilogue(tile_of(i), tmem + (uint32_t)(b * Op::NCOL), quarter, lane, xv, xq);
                afumma::fence_before_sync();
                afptx::mbar_arrive(tempty0 + 8 * b);
            }
        } else if (mytiles > 0) {
            bool ok = true;
            if constexpr (Op::UNPOOL) {
                // these warps build each tile's stage of the output gradient from
                // the pooled one once the stage is free, then arrive on its full
                // barrier: two groups of 64 threads take alternate tiles, each
                // loading its next tile's inputs before it stores this one's
                const int t = tid - 64, grp = t >> 6, tg = t & 63;
                float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                typename Op::Pooled pre;
                if (grp < mytiles) op.unpool_load(tile_of(grp), tg, pre);
                for (int g = grp; g < mytiles; g += 2) {
                    const int s = g % NS;
                    if (g >= NS && !afumma::wait_or_abort(empty0 + 8 * s, (uint32_t)(g / NS - 1) & 1u, abort)) {
                        ok = false;
                        break;
                    }
                    const typename Op::Pooled cur = pre;
                    if (g + 2 < mytiles) op.unpool_load(tile_of(g + 2), tg, pre);
                    op.unpool_store(sm + Op::RB + (size_t)s * Op::SSTAGE, tg, cur, acc);
                    afptx::fence_proxy_async();
                    afptx::mbar_arrive(full0 + 8 * s);
                }
                op.unpool_finish(t, lane, acc);
            }
            ok = afumma::wait_or_abort(tfull0, 0u, abort) && ok;
            if (!epi_sync_any(!ok || *abort)) {
                afumma::fence_after_sync();
                op.final(tmem, quarter, lane);
            }
        }
    }
    __syncthreads();
    if (tid == 0 && *abort) atomicExch(args.err, 1);
    afumma::fence_after_sync();
    if (warp == 1) afumma::tmem_dealloc(tmem, TCOLS);
}

// ------------------------------------------------------------ convolution
// Forward (POOL: + bias, ReLU, 2x2 max pool with argmax) or data gradient
// (plain store) of a 3x3 convolution over CB input channel blocks (1: the
// two-channel first layer, taps paired), N output channels, W columns.
// Packed weights (nn_tpack): step s, then its two K halves (core-matrix
// columns), then N rows of 16 bytes.
template <int CB, int N, int W, bool POOL>
struct ConvOp {
    using G = Geo<CB, W>;
    // CB == 1: the first layer's column-expanded input (one block: the 2
    // channels of columns x - 1, x, x + 1, two zeros), one unshifted copy
    static constexpr bool EXP = CB == 1;
    using H3 = Halo<CB, W, false, EXP ? 1 : 3>;
    static_assert(EXP || CB % 2 == 0, "input channel blocks: 1 or even");
    static_assert(N % 16 == 0 && N <= 128, "output channels");
    static constexpr int R = G::R, STEPS = EXP ? 2 : 9 * CB / 2;
    static constexpr uint32_t LBO_B = N / 8 * 128;  // K halves of a weight step
    static constexpr uint32_t RB = align1k(STEPS * 2 * LBO_B);
    static constexpr uint32_t SSTAGE = H3::BYTES, SLACK = 0;
    static constexpr int NCOPY = H3::NCOPY;
    static constexpr int NS = clampi(49152 / (int)SSTAGE, 2, 4);  // shallow: more blocks (epilogue warps) per SM
    static constexpr int NACC = 4, NCOL = N;
    static constexpr bool PER_TILE = true, UNPOOL = false;
    static constexpr int FULL_ARRIVALS = 1;
    struct Args {
        const __nv_bfloat16* in;  // [n][CB][H][W][8]; CB = 1: the raw input [n][H][W][2]
        const __nv_bfloat16* wp;  // packed weights, STEPS * 2 * LBO_B bytes
        const float* bias;        // [N] (POOL)
        __nv_bfloat16* out;       // POOL: [n][N/8][H/2][W/2][8]; else [n][N/8][H][W][8]
        uint8_t* idx;             // POOL: argmax | 4 if the maximum > 0, laid out as out (nullable)
        int n;  // images; every feature map is square (H = W)
        int* err;
    };
    const Args a;
    __device__ ConvOp(const Args& a_) : a(a_) {}
    __device__ int ntiles() const { return a.n * (W / R); }
    __device__ void resident(uint8_t* res, int tid) const
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.wp);
        for (int i = tid; i < (int)(STEPS * 2 * LBO_B / 16); i += kThreads)
            reinterpret_cast<uint4*>(res)[i] = __ldg(src + i);
    }
    __device__ uint32_t tx(int tile) const { return H3::tx((tile % (W / R)) * R, W); }
    __device__ void copy(int c, uint32_t st, int tile, uint32_t bar) const
    {
        const int tpi = W / R, img = tile / tpi;
        H3::copy(c, st, a.in, img, (tile - img * tpi) * R, W, bar);
    }
    __device__ void fixup(uint8_t* st, int tile, int lane) const { H3::fixup(st, (tile % (W / R)) * R, W, lane); }
    // Step s: A = the tap's copy from the tap's row, its K halves one LBO apart
    // (two channel blocks; for EXP two rows dy); B = the step's weights.
    __device__ void mma(uint32_t st, uint32_t res, uint32_t tmem, int) const
    {
        constexpr uint32_t idesc = afumma::idesc_bf16(128, N, 0, 0);
#pragma unroll
        for (int s = 0; s < STEPS; s++) {
            uint32_t a0, lbo;
            if constexpr (EXP) {
                // rows (0, 1), then (1, 2) with zero weights in the first half
                a0 = st + s * W * 16;
                lbo = W * 16;
            } else {
                const int t = s / (CB / 2), j = s % (CB / 2);
                a0 = st + H3::plane(t % 3, 2 * j) + (t / 3) * W * 16;
                lbo = G::PLANE;
            }
            afumma::mma_bf16(tmem, afumma::smem_desc(a0, lbo, 128),
                             afumma::smem_desc(res + (uint32_t)s * 2 * LBO_B, LBO_B, 128), idesc, s != 0);
        }
    }
    __device__ void final(uint32_t, int, int) const {}
    // Thread = tile row r = 32 quarter + lane, pixel (y0 + r / W, r % W).
    __device__ void epilogue(int tile, uint32_t tmem, int quarter, int lane, float* xv, uint32_t* xq) const
    {
        const int tpi = W / R, img = tile / tpi, y0 = (tile - img * tpi) * R;
        const int r = 32 * quarter + lane, yl = r / W, x = r % W;
        const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16);
        if constexpr (!POOL) {
            const int64_t plane = (int64_t)W * W, pix = (int64_t)(y0 + yl) * W + x;
#pragma unroll 1
            for (int c0 = 0; c0 < N; c0 += 16) {
                uint32_t v[16];
                afumma::ld_32x32b_x16(taddr + (uint32_t)c0, v);
                afumma::wait_ld();
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const uint32_t* u = v + 8 * h;
                    const uint4 o = make_uint4(pack_bf16(__uint_as_float(u[0]), __uint_as_float(u[1])),
                                               pack_bf16(__uint_as_float(u[2]), __uint_as_float(u[3])),
                                               pack_bf16(__uint_as_float(u[4]), __uint_as_float(u[5])),
                                               pack_bf16(__uint_as_float(u[6]), __uint_as_float(u[7])));
                    *reinterpret_cast<uint4*>(a.out + (((int64_t)img * (N / 8) + c0 / 8 + h) * plane + pix) * 8) = o;
                }
            }
        } else if (a.idx) {
            pool_epilogue<true>(img, y0, yl, x, quarter, lane, taddr, xv, xq);
        } else {
            pool_epilogue<false>(img, y0, yl, x, quarter, lane, taddr, xv, xq);
        }
    }

    // Inference: the same pooling on the bf16-rounded values, two channels a
    // word (rounding to nearest is monotone, so the maximum of the rounded
    // values is the rounded maximum, and the ReLU of it likewise: the same
    // bf16 outputs as pooling in fp32 and rounding once).  m: this lane's 16
    // biased channels of the chunk c0.
    __device__ void pool_infer(const float (&m)[16], int c0, int img, int64_t po, int64_t oplane, bool top, bool odd,
                               int slot, uint4* xv4) const
    {
        uint32_t q[8];
#pragma unroll
        for (int i = 0; i < 8; i++) q[i] = pack_bf16(m[2 * i], m[2 * i + 1]);
        // the even column keeps channel pairs 0-3, the odd one 4-7
        __nv_bfloat162 h[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const uint32_t keep = odd ? q[i + 4] : q[i], give = odd ? q[i] : q[i + 4];
            const uint32_t other = __shfl_xor_sync(0xffffffffu, give, 1);
            h[i] = __hmax2(*reinterpret_cast<const __nv_bfloat162*>(&keep),
                           *reinterpret_cast<const __nv_bfloat162*>(&other));
        }
        if constexpr (W == 16) {
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const uint32_t o = __shfl_xor_sync(0xffffffffu, *reinterpret_cast<const uint32_t*>(&h[i]), 16);
                h[i] = __hmax2(h[i], *reinterpret_cast<const __nv_bfloat162*>(&o));
            }
        } else {
            if (!top) xv4[2 * slot] = *reinterpret_cast<const uint4*>(h);
            epi_sync();
            if (top) {
                const uint4 lo = xv4[2 * slot];
                const __nv_bfloat162* l2 = reinterpret_cast<const __nv_bfloat162*>(&lo);
#pragma unroll
                for (int i = 0; i < 4; i++) h[i] = __hmax2(h[i], l2[i]);
            }
            epi_sync();
        }
        if (top) {
            const __nv_bfloat162 z = __float2bfloat162_rn(0.f);
#pragma unroll
            for (int i = 0; i < 4; i++) h[i] = __hmax2(h[i], z);
            const int64_t e0 = (((int64_t)img * (N / 8) + c0 / 8 + (odd ? 1 : 0)) * oplane + po) * 8;
            *reinterpret_cast<uint4*>(a.out + e0) = *reinterpret_cast<const uint4*>(h);
        }
    }

    // Bias, 2 x 2 max pool and ReLU (pooled before the ReLU: it commutes with
    // the maximum; where the maximum is positive the argmax is the ReLU
    // outputs' one, elsewhere no gradient is routed) and, in training, the
    // argmax byte.  Per chunk of 16 channels the two lanes of a horizontal
    // pixel pair split the chunk (the even column keeps channels 0-7, the odd
    // one 8-15), so every later step handles 8 channels per lane; the upper
    // row of a window finishes it, the row below coming through a lane
    // shuffle (W = 16: 16 lanes on) or, from another warp, through shared
    // memory (slot 32 p + lane of warp pair p, 8 floats and the row's bits).
    template <bool TRAIN>
    __device__ void pool_epilogue(int img, int y0, int yl, int x, int quarter, int lane, uint32_t taddr, float* xv,
                                  uint32_t* xq) const
    {
        const int Ho = W / 2, Wo = W / 2;
        const bool top = (yl & 1) == 0, odd = (x & 1) != 0;
        const int64_t po = (int64_t)(y0 / 2 + (yl >> 1)) * Wo + (x >> 1), oplane = (int64_t)Ho * Wo;
        const int slot = 32 * (W == 64 ? (quarter & 1) : (quarter >> 1)) + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t v[16];
            afumma::ld_32x32b_x16(taddr + (uint32_t)c0, v);
            afumma::wait_ld();
            float m[16];
            const float4* bv = reinterpret_cast<const float4*>(a.bias + c0);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float4 b4 = __ldg(bv + k);
                m[4 * k] = __uint_as_float(v[4 * k]) + b4.x;
                m[4 * k + 1] = __uint_as_float(v[4 * k + 1]) + b4.y;
                m[4 * k + 2] = __uint_as_float(v[4 * k + 2]) + b4.z;
                m[4 * k + 3] = __uint_as_float(v[4 * k + 3]) + b4.w;
            }
            if constexpr (!TRAIN) {
                pool_infer(m, c0, img, po, oplane, top, odd, slot, reinterpret_cast<uint4*>(xv));
                continue;
            }
            // the pair's row maximum of this lane's 8 channels; hx bit i: the
            // right pixel strictly larger (a tie keeps the left, earlier in raster order)
            float h[8];
            uint32_t hx = 0u;
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const float keep = odd ? m[i + 8] : m[i], give = odd ? m[i] : m[i + 8];
                const float other = __shfl_xor_sync(0xffffffffu, give, 1);
                if (TRAIN) hx |= ((odd ? keep > other : other > keep) ? 1u : 0u) << i;
                h[i] = fmaxf(keep, other);
            }
            // the row below: vy bit i where it is strictly larger; hx_low its hx
            uint32_t vy = 0u, hx_low = 0u;
            if constexpr (W == 16) {
                if (TRAIN) hx_low = __shfl_xor_sync(0xffffffffu, hx, 16);
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const float o = __shfl_xor_sync(0xffffffffu, h[i], 16);
                    if (TRAIN) vy |= (o > h[i] ? 1u : 0u) << i;
                    h[i] = fmaxf(h[i], o);
                }
            } else {
                float4* sv = reinterpret_cast<float4*>(xv) + 2 * slot;
                if (!top) {
                    sv[0] = make_float4(h[0], h[1], h[2], h[3]);
                    sv[1] = make_float4(h[4], h[5], h[6], h[7]);
                    if (TRAIN) xq[slot] = hx;
                }
                epi_sync();
                if (top) {
                    const float4 l0 = sv[0], l1 = sv[1];
                    const float lo[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        if (TRAIN) vy |= (lo[i] > h[i] ? 1u : 0u) << i;
                        h[i] = fmaxf(h[i], lo[i]);
                    }
                    if (TRAIN) hx_low = xq[slot];
                }
                epi_sync();
            }
            if (top) {
                const int64_t e0 = (((int64_t)img * (N / 8) + c0 / 8 + (odd ? 1 : 0)) * oplane + po) * 8;
                *reinterpret_cast<uint4*>(a.out + e0) =
                    make_uint4(pack_bf16(fmaxf(h[0], 0.f), fmaxf(h[1], 0.f)), pack_bf16(fmaxf(h[2], 0.f), fmaxf(h[3], 0.f)),
                               pack_bf16(fmaxf(h[4], 0.f), fmaxf(h[5], 0.f)), pack_bf16(fmaxf(h[6], 0.f), fmaxf(h[7], 0.f)));
                if (TRAIN) {
                    // argmax in raster order: (lower row won ? 2 + its column : this row's column), | 4 if positive
                    uint32_t w2[2] = {0u, 0u};
#pragma unroll
                    for (int k = 0; k < 8; k++) {
                        const uint32_t q = ((vy >> k) & 1u) ? 2u | ((hx_low >> k) & 1u) : (hx >> k) & 1u;
                        w2[k >> 2] |= (q | (h[k] > 0.f ? 4u : 0u)) << (8 * (k & 3));
                    }
                    *reinterpret_cast<uint2*>(a.idx + e0) = make_uint2(w2[0], w2[1]);
                }
            }
        }
    }
};


// ------------------------------------------------------------ weight gradient
// dW[o][t][i] += sum over the block's tiles of dZ[p][o] X[p + t][i], with ZB
// output channel blocks (COUT = 8 ZB) and CB input channel blocks (1: the
// two-channel first layer).  A stage holds the tile's dZ rows (R rows of every
// block, one bulk copy per block) and the three shifted copies of X.  A
// (dZ^T) has 128 rows of which COUT are real: the others read up to 16
// channel blocks from the stage's start (past the ring's end for the last
// stage: the zeroed slack) and their results are never read.  Per 16 pixels
// of K:
//   TAPN: one MMA per input block whose N columns are the taps: with the
//     block's three copies back to back, tap (dy, dx) starts (dy + (R + 2) dx)
//     rows after the first, so N = 8 NJ columns (NJ = 2 (R + 2) + 3 rounded up
//     to even) at a stride of one row take every tap in one MMA (the columns
//     of dy >= 3 are read and dropped); A is read once for all taps.  The
//     first layer (CB = 1) reads its column-expanded input unshifted: N = 32
//     columns, rows dy = 0 .. 3, each 8 channels (dx, c) for dx < 3, c < 2.
//   else: one MMA per tap, N = the block's channels.
template <int CB, int ZB, int W, bool TAPN, bool UNPOOL_ = false>
struct WgradOp {
    using G = Geo<CB, W>;
    using H3 = Halo<CB, W, (TAPN && CB > 1), (CB == 1 ? 1 : 3)>;
    static_assert(CB == 1 || CB % 2 == 0, "input channel blocks: 1 or even");
    static_assert(TAPN || CB >= 2, "the per-tap form needs N = 8 CB >= 16");
    static constexpr int R = G::R, CIN = CB == 1 ? 2 : CB * 8, COUT = ZB * 8;
    static constexpr int NJ = CB == 1 ? 4 : (2 * (R + 2) + 3 + 1) / 2 * 2;
    static constexpr int NPM = TAPN ? 8 * NJ : CB * 8;  // N of one MMA
    static constexpr int NMMA = TAPN ? CB : 9;          // MMAs per K step
    static_assert(NPM % 16 == 0 && NPM <= 256, "MMA width");
    static_assert(COUT <= 128, "output channels");
    static constexpr uint32_t PLANE_Z = (uint32_t)R * W * 16, ZREG = align1k(PLANE_Z * ZB);
    static constexpr uint32_t RB = 0, SSTAGE = ZREG + H3::BYTES;
    // UNPOOL: dZ is not read from memory but built in each stage from the
    // pooled gradient dP and the argmax bytes (the pooling layer's backward
    // pass), by the epilogue warps, which are otherwise idle until the end
    static constexpr bool UNPOOL = UNPOOL_;
    static constexpr int FULL_ARRIVALS = UNPOOL ? 1 + 64 : 1;
    static constexpr int NCOPY = H3::NCOPY + (UNPOOL ? 0 : ZB);
    // SWAP (taps along N with input blocks of 8 channels, i.e. layer 1): the
    // roles turn around, A = the block's copies (M = 8 NJ = 128 rows: tap row
    // shift j, channel), B = dZ^T (N = COUT), so the MMA is 128 x COUT instead
    // of 128 x 8 NJ of which only COUT rows are real, and reads no slack
    static constexpr bool SWAP = TAPN && CB > 1;
    static_assert(!SWAP || (8 * NJ == 128 && COUT % 16 == 0), "swapped weight-gradient shape");
    static constexpr uint32_t SLACK = !SWAP && 16 * PLANE_Z > SSTAGE ? 16 * PLANE_Z - SSTAGE : 0;
    static constexpr int NS = clampi(65536 / (int)SSTAGE, 2, 4);
    static constexpr int NACC = 1, NCOL = NMMA * (SWAP ? COUT : NPM);
    static_assert(NCOL <= 512, "tensor-memory columns");
    static constexpr bool PER_TILE = false;
    struct Args {
        const __nv_bfloat16* x;   // [n][CB][H][W][8]; CB = 1: the raw input [n][H][W][2]
        const __nv_bfloat16* dz;  // [n][ZB][H][W][8] (not UNPOOL)
        float* grad;              // [COUT][9][CIN], accumulated
        int n;                    // images; every feature map is square (H = W)
        int* err;
        const __nv_bfloat16* dp;  // UNPOOL: pooled gradient [n][ZB][H/2][W/2][8]
        const uint8_t* idx;       // UNPOOL: argmax 0..3 | 4 if positive, laid out as dp
        float* db;                // UNPOOL: [COUT] bias gradient (the sum of dZ), accumulated
    };
    const Args a;
    __device__ WgradOp(const Args& a_) : a(a_) {}
    __device__ int ntiles() const { return a.n * (W / R); }
    __device__ void resident(uint8_t*, int) const {}
    __device__ uint32_t tx(int tile) const
    {
        return H3::tx((tile % (W / R)) * R, W) + (UNPOOL ? 0u : ZB * PLANE_Z);
    }
    // UNPOOL: thread tg (< 64) of a group of the epilogue warps handles item
    // tg of a tile, (pooled pixel tg / ZB of the tile's R / 2 pooled rows,
    // block tg % ZB): its gradient goes to the window's argmax where the
    // maximum was positive, zeros to the other three pixels; acc sums the
    // routed values of block tg % ZB (the bias gradient).
    struct Pooled {
        uint4 v;   // 8 channels of the pooled gradient
        uint2 ix;  // their argmax bytes
    };
    static constexpr int ITEMS = ZB * (R / 2) * (W / 2);
    static_assert(!UNPOOL || ITEMS == 64, "one item per thread of a 64-thread group");
    __device__ void unpool_load(int tile, int tg, Pooled& p) const
    {
        const int tpi = W / R, img = tile / tpi, y0 = (tile - img * tpi) * R;
        const int zb = tg % ZB, pp = tg / ZB, pr = pp / (W / 2), xo = pp - pr * (W / 2);
        const int64_t e = ((((int64_t)img * ZB + zb) * (W / 2) + y0 / 2 + pr) * (W / 2) + xo) * 8;
        p.v = __ldg(reinterpret_cast<const uint4*>(a.dp + e));
        p.ix = __ldg(reinterpret_cast<const uint2*>(a.idx + e));
    }
    __device__ void unpool_store(uint8_t* st, int tg, const Pooled& p, float (&acc)[8]) const
    {
        const int zb = tg % ZB, pp = tg / ZB, pr = pp / (W / 2), xo = pp - pr * (W / 2);
        const uint16_t* vv = reinterpret_cast<const uint16_t*>(&p.v);
        const uint8_t* ii = reinterpret_cast<const uint8_t*>(&p.ix);
#pragma unroll
        for (int j = 0; j < 8; j++)
            if (ii[j] & 4) acc[j] += __bfloat162float(__ushort_as_bfloat16(vv[j]));
#pragma unroll
        for (int q = 0; q < 4; q++) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t lo = ii[2 * j] == (uint8_t)(4 | q) ? vv[2 * j] : 0u;
                const uint32_t hi = ii[2 * j + 1] == (uint8_t)(4 | q) ? vv[2 * j + 1] : 0u;
                w[j] = lo | (hi << 16);
            }
            const int r = 2 * pr + (q >> 1), x = 2 * xo + (q & 1);
            *reinterpret_cast<uint4*>(st + zb * PLANE_Z + (r * W + x) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
    // The bias gradient: the lanes of a warp with one block reduce, then one
    // atomic per channel and warp.
    __device__ void unpool_finish(int t, int lane, float (&acc)[8]) const
    {
#pragma unroll
        for (int j = 0; j < 8; j++) {
#pragma unroll
            for (int o = 16; o >= ZB; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
            if (lane < ZB) atomicAdd(a.db + (t % ZB) * 8 + j, acc[j]);  // t % ZB = lane % ZB
        }
    }
    // copies 0 .. 3 CB - 1: the shifted copies of X; then one per dZ block
    __device__ void copy(int c, uint32_t st, int tile, uint32_t bar) const
    {
        const int tpi = W / R, img = tile / tpi, y0 = (tile - img * tpi) * R;
        if (c < H3::NCOPY) {
            H3::copy(c, st + ZREG, a.x, img, y0, W, bar);
        } else {
            const int zb = c - H3::NCOPY;
            afptx::bulk_g2s(st + zb * PLANE_Z, a.dz + (((int64_t)img * ZB + zb) * W + y0) * W * 8, PLANE_Z, bar);
        }
    }
    __device__ void fixup(uint8_t* st, int tile, int lane) const
    {
        H3::fixup(st + ZREG, (tile % (W / R)) * R, W, lane);
    }
    // K step ks = pixels 16 ks .. 16 ks + 15 of the tile; MN-major operands:
    // core matrices of 8 pixels (K, 128 bytes apart) by 8 channels (M / N).
    __device__ void mma(uint32_t st, uint32_t, uint32_t tmem, int g) const
    {
        const uint32_t xs = st + ZREG;
        if constexpr (SWAP) {
            constexpr uint32_t idesc = afumma::idesc_bf16(128, COUT, 1, 1);
#pragma unroll 1
            for (int ks = 0; ks < 8; ks++) {
                const uint64_t db = afumma::smem_desc(st + ks * 256, 128, PLANE_Z);
#pragma unroll
                for (int k = 0; k < NMMA; k++)
                    afumma::mma_bf16(tmem + (uint32_t)(k * COUT),
                                     afumma::smem_desc(xs + H3::plane(0, k) + ks * 256, 128, W * 16), db, idesc,
                                     (g | ks) != 0);
            }
            return;
        }
        constexpr uint32_t idesc = afumma::idesc_bf16(128, NPM, 1, 1);
#pragma unroll 1
        for (int ks = 0; ks < 8; ks++) {
            const uint64_t da = afumma::smem_desc(st + ks * 256, 128, PLANE_Z);
#pragma unroll
            for (int k = 0; k < NMMA; k++) {
                uint32_t b0, sbo;
                if constexpr (TAPN) {
                    b0 = xs + H3::plane(0, k);  // block k: its taps one row apart along N
                    sbo = W * 16;
                } else {
                    b0 = xs + H3::plane(k % 3, 0) + (k / 3) * W * 16;  // tap k, N = the blocks
                    sbo = G::PLANE;
                }
                afumma::mma_bf16(tmem + (uint32_t)(k * NPM), da, afumma::smem_desc(b0 + ks * 256, 128, sbo), idesc,
                                 (g | ks) != 0);
            }
        }
    }
    __device__ void epilogue(int, uint32_t, int, int, float*, uint32_t*) const {}
    // Row o = 32 quarter + lane of the accumulator: its columns into grad.
    __device__ void final(uint32_t tmem, int quarter, int lane) const
    {
        if constexpr (SWAP) {
            // row m = 32 quarter + lane: row shift j = m / 8 of a block's copies
            // (tap dy = j % (R + 2), dx = j / (R + 2)), channel m % 8; columns:
            // block k's COUT outputs
            const int m = 32 * quarter + lane, j = m >> 3, dx = j / (R + 2), dy = j - dx * (R + 2);
            const bool real = dy < 3 && dx < 3;
            const int t = 3 * dy + dx;
            const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16);
#pragma unroll 1
            for (int k = 0; k < NMMA; k++)
#pragma unroll 1
                for (int c0 = 0; c0 < COUT; c0 += 16) {
                    uint32_t v[16];
                    afumma::ld_32x32b_x16(taddr + (uint32_t)(k * COUT + c0), v);
                    afumma::wait_ld();
                    if (!real) continue;
                    const int i = 8 * k + (m & 7);
#pragma unroll
                    for (int jj = 0; jj < 16; jj++)
                        atomicAdd(a.grad + ((int64_t)(c0 + jj) * 9 + t) * CIN + i, __uint_as_float(v[jj]));
                }
            return;
        }
        if (32 * quarter >= COUT) return;  // warp-uniform: no real rows in this quarter
        const int o = 32 * quarter + lane;
        const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < NCOL; c0 += 16) {
            uint32_t v[16];
            afumma::ld_32x32b_x16(taddr + (uint32_t)c0, v);
            afumma::wait_ld();
            if (o >= COUT) continue;
#pragma unroll
            for (int jj = 0; jj < 16; jj++) {
                const int col = c0 + jj;
                int t, i;
                if constexpr (CB == 1) {
                    const int dy = col >> 3, dx = (col & 7) >> 1;
                    i = col & 1;
                    if (dy >= 3 || dx >= 3) continue;
                    t = 3 * dy + dx;
                } else if constexpr (TAPN) {
                    const int k = col / NPM, r = col - k * NPM, j = r >> 3, dx = j / (R + 2), dy = j - dx * (R + 2);
                    i = 8 * k + (r & 7);
                    if (dy >= 3 || dx >= 3 || i >= CIN) continue;
                    t = 3 * dy + dx;
                } else {
                    t = col / NPM;
                    i = col - t * NPM;
                }
                atomicAdd(a.grad + ((int64_t)o * 9 + t) * CIN + i, __uint_as_float(v[jj]));
            }
        }
    }
};

// ------------------------------------------------------------ weights and input
// Packed B operand of ConvOp, element e = ((s * 2 + kc) * nrows + row) * 8 + k:
// step s, K half kc, row (an output channel of the operation), channel k of
// the K half's block.  Forward: rows o, K = (tap t, input channel i).  Data
// gradient: rows i, K = (tap t, o) with the taps flipped, W'[i][t][o] =
// W[o][8 - t][i].  cbk = channel blocks of K per tap (1: the first layer's
// column-expanded input, two K steps of rows (0, 1) and (1, 2), the repeated
// row 1 with zero weights).
__global__ void k_tpack(const float* __restrict__ w, int cin, int cout, int cbk, int nrows, int dgrad, int total,
                        __nv_bfloat16* __restrict__ out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int k = e & 7, row = (e >> 3) % nrows, kc = (e / (8 * nrows)) & 1, s = e / (16 * nrows);
    int t, c;
    if (cbk == 1) {
        // column-expanded input: K half kc of step s is row dy = s + kc (step 1's
        // first half repeats row 1 with zero weights), channel k = (dx, c)
        const int dy = s + kc;
        t = (s == 1 && kc == 0) || k >= 6 ? -1 : 3 * dy + (k >> 1);
        c = k & 1;
    } else {
        t = s / (cbk / 2);
        c = (2 * (s % (cbk / 2)) + kc) * 8 + k;
    }
    float v = 0.f;
    if (t >= 0) {
        if (!dgrad && c < cin) v = w[((int64_t)row * 9 + t) * cin + c];
        if (dgrad && c < cout) v = w[((int64_t)c * 9 + (8 - t)) * cin + row];
    }
    out[e] = __float2bfloat16(v);
}

// ------------------------------------------------------------ host side
template <class Op>
constexpr size_t smem_bytes()
{
    return 1024 + (size_t)Op::RB + (size_t)Op::NS * Op::SSTAGE + Op::SLACK;
}

// Resident blocks of Op per device (computed once per device, under a lock:
// model calls may come from several host threads).
template <class Op>
int resident_blocks(int dev, int* out)
{
    static std::mutex mu;
    static std::map<int, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) {
        *out = it->second;
        return AF_OK;
    }
    const size_t smem = smem_bytes<Op>();
    AF_CUDA(cudaFuncSetAttribute(k_tconv<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    AF_CUDA(cudaFuncSetAttribute(k_tconv<Op>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    int nsm = 0, per_sm = 0, smem_sm = 0;
    cudaFuncAttributes fa;
    AF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    AF_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    AF_CUDA(cudaFuncGetAttributes(&fa, k_tconv<Op>));
    AF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tconv<Op>, kThreads, smem));
    // by shared memory (1 KB reserved per block), at most the 512 tensor-memory
    // columns' share; the occupancy query's answer when it is larger
    const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);
    const int by_tmem = 512 / pow2_cols(Op::NACC * Op::NCOL);
    int b = by_smem > per_sm ? by_smem : per_sm;
    if (b > by_tmem) b = by_tmem;
    *out = cache[dev] = (b < 1 ? 1 : b) * nsm;
    return AF_OK;
}

template <class Op>
int launch(const typename Op::Args& a, int ntiles, cudaStream_t s, const char* what)
{
    if (ntiles <= 0) return AF_OK;
    int dev = 0, blocks = 0;
    AF_CUDA(cudaGetDevice(&dev));
    if (int rc = resident_blocks<Op>(dev, &blocks)) return rc;
    const int grid = ntiles < blocks ? ntiles : blocks;
    k_tconv<Op><<<grid, kThreads, smem_bytes<Op>(), s>>>(a);
    return af_cuda_check(cudaGetLastError(), what);
}

// The classifier's layers: input channels, output channels, width (= height).
constexpr int kCin[3] = {2, 16, 32}, kCout[3] = {16, 32, 64}, kW[3] = {64, 32, 16};

using Fwd0 = ConvOp<1, 16, 64, true>;
using Fwd1 = ConvOp<2, 32, 32, true>;
using Fwd2 = ConvOp<4, 64, 16, true>;
using Dg1 = ConvOp<4, 16, 32, false>;
using Dg2 = ConvOp<8, 32, 16, false>;
using Wg0 = WgradOp<1, 2, 64, true>;
using Wg0u = WgradOp<1, 2, 64, true, true>;  // layer 0's output gradient built from the pooled one
using Wg1 = WgradOp<2, 4, 32, true>;
using Wg2 = WgradOp<4, 8, 16, false>;

}  // namespace

size_t nn_tpack_bytes(int layer, int dgrad)
{
    if (!dgrad) return layer == 0 ? Fwd0::STEPS * 2 * Fwd0::LBO_B : layer == 1 ? Fwd1::STEPS * 2 * Fwd1::LBO_B
                                                                               : Fwd2::STEPS * 2 * Fwd2::LBO_B;
    return layer == 1 ? Dg1::STEPS * 2 * Dg1::LBO_B : layer == 2 ? Dg2::STEPS * 2 * Dg2::LBO_B : 0;
}

int nn_tpack(int layer, int dgrad, const float* w, __nv_bfloat16* out, cudaStream_t s)
{
    if (layer < 0 || layer > 2 || (dgrad && layer == 0)) return af_set_error(AF_EINVAL, "conv pack: layer %d", layer);
    const int cin = kCin[layer], cout = kCout[layer];
    const int cbk = dgrad ? cout / 8 : (cin < 8 ? 1 : cin / 8), nrows = dgrad ? cin : cout;  // cbk 1: expanded
    const int total = (int)(nn_tpack_bytes(layer, dgrad) / 2);
    k_tpack<<<(total + 255) / 256, 256, 0, s>>>(w, cin, cout, cbk, nrows, dgrad, total, out);
    return af_cuda_check(cudaGetLastError(), "conv pack");
}

int nn_tconv_fwd(int layer, const __nv_bfloat16* x, int n, const __nv_bfloat16* wp, const float* bias,
                 __nv_bfloat16* out, uint8_t* idx, int* err, cudaStream_t s)
{
    if (layer < 0 || layer > 2 || n < 1 || !x || ((uintptr_t)x & 15) || ((uintptr_t)out & 15) ||
        ((uintptr_t)idx & 15) || ((uintptr_t)bias & 15))
        return af_set_error(AF_EINVAL, "conv forward: layer %d / alignment", layer);
    const int W = kW[layer], tiles = n * (W / (128 / W));
#define AF_TF(L, Op)                                                  \
    if (layer == L) {                                                 \
        typename Op::Args a{x, wp, bias, out, idx, n, err};        \
        return launch<Op>(a, tiles, s, "conv forward (tcgen05)");     \
    }
    AF_TF(0, Fwd0)
    AF_TF(1, Fwd1)
    AF_TF(2, Fwd2)
#undef AF_TF
    return AF_OK;
}

int nn_tconv_dgrad(int layer, const __nv_bfloat16* dz, int n, const __nv_bfloat16* wp, __nv_bfloat16* dx, int* err,
                   cudaStream_t s)
{
    if (layer < 1 || layer > 2 || n < 1 || !dz || ((uintptr_t)dz & 15) || ((uintptr_t)dx & 15))
        return af_set_error(AF_EINVAL, "conv data gradient: layer %d / alignment", layer);
    const int W = kW[layer], tiles = n * (W / (128 / W));
#define AF_TD(L, Op)                                                      \
    if (layer == L) {                                                     \
        typename Op::Args a{dz, wp, nullptr, dx, nullptr, n, err};     \
        return launch<Op>(a, tiles, s, "conv data gradient (tcgen05)");   \
    }
    AF_TD(1, Dg1)
    AF_TD(2, Dg2)
#undef AF_TD
    return AF_OK;
}

int nn_tconv_wgrad(int layer, const __nv_bfloat16* dz, const __nv_bfloat16* x, int n, float* grad, int* err,
                   cudaStream_t s)
{
    if (layer < 0 || layer > 2 || n < 1 || !x || !dz || ((uintptr_t)x & 15) || ((uintptr_t)dz & 15))
        return af_set_error(AF_EINVAL, "conv weight gradient: layer %d / alignment", layer);
    const int W = kW[layer], tiles = n * (W / (128 / W));
#define AF_TW(L, Op)                                                      \
    if (layer == L) {                                                     \
        typename Op::Args a{x, dz, grad, n, err, nullptr, nullptr, nullptr}; \
        return launch<Op>(a, tiles, s, "conv weight gradient (tcgen05)"); \
    }
    AF_TW(0, Wg0)
    AF_TW(1, Wg1)
    AF_TW(2, Wg2)
#undef AF_TW
    return AF_OK;
}

int nn_tconv_wgrad_unpool(const __nv_bfloat16* dp, const uint8_t* idx, const __nv_bfloat16* x, int n, float* grad,
                          float* db, int* err, cudaStream_t s)
{
    if (n < 1 || !x || !dp || !idx || !db || ((uintptr_t)x & 15) || ((uintptr_t)dp & 15) || ((uintptr_t)idx & 7))
        return af_set_error(AF_EINVAL, "conv weight gradient (unpool): argument / alignment");
    const int W = kW[0], tiles = n * (W / (128 / W));
    typename Wg0u::Args a{x, nullptr, grad, n, err, dp, idx, db};
    return launch<Wg0u>(a, tiles, s, "conv weight gradient with pool backward (tcgen05)");
}
