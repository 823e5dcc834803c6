// conv_umma.cu -- the classifier's contractions on the 5th-generation tensor
// cores (tcgen05.mma kind::f16: bf16 operands, fp32 accumulators in tensor
// memory).  The classifier replaces the paper's YOLO detector (Sec. 2.5);
// its 3x3 convolutions are implicit GEMMs, so no im2col matrix is ever
// written:
//
//   forward  Z[p][o]   = sum_{t,i} X[p + t][i] W[o][t][i]      M = pixels, N = Cout, K = 9 Cin
//            with bias, ReLU and the 2x2 max pool in the epilogue (pooled
//            bf16 activations and the argmax out; the fp32 Z never leaves
//            tensor memory)
//   dgrad    dX[p][i]  = sum_{t,o} dZ[p - t][o] W[o][t][i]     M = pixels, N = Cin,  K = 9 Cout
//   wgrad    dW[o][t][i] = sum_p dZ[p][o] X[p + t][i]          M = Cout,   N = 9 Cin, K = pixels (split)
//
// plus a plain GEMM C = A B (af_nn_gemm) in the four operand layouts.
//
// One pipelined kernel serves every operation: 128 threads stage operand
// tiles with 16-byte (4-byte for 2-channel inputs) cp.async copies, zero
// filled outside the image or the matrix, straight into the no-swizzle
// canonical layout of umma.cuh (the im2col gather is the copy's address);
// weights that every tile uses stay resident in shared memory; thread 0
// issues the MMAs of a stage and commits them onto the stage's mbarrier,
// which frees the stage for the copies NS - 2 stages later; after a tile's
// last stage every warp reads its 32 tensor-memory lanes (rows) back with
// tcgen05.ld for the epilogue.  Every mbarrier wait is bounded: a wait that
// runs out raises the caller's error flag and the kernel leaves cleanly.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>

#include "internal.h"
#include "nn.h"
#include "ptx.cuh"
#include "umma.cuh"

namespace {

// producer warps 0-3, MMA warp 4, epilogue warps 5-8
constexpr int kProd = 128, kEpi = 128, kBlock = kProd + 32 + kEpi;

// cp.async of 16 (4) bytes through L1 (a 3x3 gather reads each input pixel up
// to nine times); `bytes` < size zero-fills the rest (0: no read)
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp4(uint32_t dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Byte offset of a 16-byte chunk inside a tile of R rows (R a multiple of 8),
// core matrix (row group, k group) at ((k group) * R/8 + row group) * 128:
//   K-major: row r, k group kg (8 consecutive k)  -> + (r % 8) * 16
//   MN-major: row group rg (8 consecutive rows), k -> + (k % 8) * 16
// so the K-direction core-matrix stride is R/8 * 128 bytes, the row-direction 128.
__device__ __forceinline__ uint32_t kmaj_off(int r, int kg, int R)
{
    return ((uint32_t)(kg * (R >> 3) + (r >> 3)) << 7) + ((uint32_t)(r & 7) << 4);
}
__device__ __forceinline__ uint32_t mnmaj_off(int rg, int k, int R)
{
    return ((uint32_t)((k >> 3) * (R >> 3) + rg) << 7) + ((uint32_t)(k & 7) << 4);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

constexpr int pow2_cols(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : n <= 256 ? 256 : 512; }

// ------------------------------------------------------------ the pipeline
// Warp-specialised: warps 0-3 produce (stage operand tiles with cp.async),
// warp 4 issues the MMAs (one elected thread), warps 5-8 run the epilogue
// (warp w reads tensor-memory lanes 32 (w % 4) ..).  Stages pass between them
// through mbarriers:
//   full[s]   128 producer arrivals: the stage's copies have landed and were
//             made visible to the tensor cores (each producer thread waits for
//             its own copies of a stage L steps later, fences, arrives)
//   empty[s]  one tcgen05.commit: the MMAs reading the stage are done
//   tfull[b]  one tcgen05.commit: accumulator b holds a finished tile
//   tempty[b] 128 epilogue arrivals: accumulator b has been read
// NACC accumulators of Op::NCOL columns each alternate between tiles, so the
// epilogue of one tile overlaps the MMAs of the next.
// Op provides: NS (stages), LAG, NACC, NCOL, SA / SB (bytes of a stage's A / B
// tile), RB (resident bytes), ntiles(), nkb(), resident(), stage(), mma(),
// epilogue().
// A producer thread arrives for a stage Op::LAG steps after issuing its
// copies (LAG stages of its copies in flight, LAG < NS).

// One poll of an mbarrier phase that suspends the thread for at most
// `hint_ns` (the hardware returns earlier when the phase completes).
__device__ __forceinline__ bool mbar_try_wait_hint(uint32_t bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for a phase with short suspensions (a pipeline step is microseconds),
// giving up after kWaitNs of wall time or when another thread gave up; a wait
// that gives up raises the block's abort flag.
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort)
{
    if (mbar_try_wait_hint(bar, parity, 200u)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t i = 1;; i++) {
        if (mbar_try_wait_hint(bar, parity, 200u)) return true;
        if ((i & 15) == 0) {
            if (*abort) return false;
            if (globaltimer_ns() - t0 > kWaitNs) break;
        }
    }
    *abort = 1;
    return false;
}

template <class Op>
__global__ void __launch_bounds__(kBlock) k_umma(const typename Op::Args args)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t bars[2 * Op::NS + 2 * Op::NACC];
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    constexpr int NS = Op::NS, NACC = Op::NACC, kLag = Op::LAG;
    constexpr uint32_t SSTAGE = Op::SA + Op::SB;
    constexpr uint32_t TCOLS = pow2_cols(NACC * Op::NCOL);
    static_assert(kLag < NS, "the producer must be able to run LAG stages ahead");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const Op op(args);
    const int ntiles = op.ntiles(), nkb = op.nkb();
    const int mytiles = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const int G = mytiles * nkb;
    uint8_t* stages = smem + Op::RB;
    const uint32_t full0 = afptx::smem_addr(bars), empty0 = full0 + 8 * NS, tfull0 = empty0 + 8 * NS,
                   tempty0 = tfull0 + 8 * NACC;
    volatile int* abort = &abort_flag;

    if (tid == 0) {
        for (int s = 0; s < NS; s++) {
            afptx::mbar_init(full0 + 8 * s, kProd);
            afptx::mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < NACC; b++) {
            afptx::mbar_init(tfull0 + 8 * b, 1);
            afptx::mbar_init(tempty0 + 8 * b, kEpi);
        }
        abort_flag = 0;
        afptx::fence_mbar_init();
    }
    if (warp == 4) {
        afumma::tmem_alloc(afptx::smem_addr(&tslot), TCOLS);
        afumma::tmem_relinquish();
    }
    afumma::fence_before_sync();
    __syncthreads();
    afumma::fence_after_sync();
    const uint32_t tmem = tslot;
    auto tile_of = [&](int g) { return (int)blockIdx.x + (g / nkb) * (int)gridDim.x; };

    if (warp < 4) {
        // ---------------- producers
        op.resident(smem, tid);  // joins the copies of step 0
        int g = 0;
        for (; g < G; g++) {
            const int s = g % NS;
            if (g >= NS && !wait_or_abort(empty0 + 8 * s, (uint32_t)(g / NS - 1) & 1u, abort)) break;
            op.stage(stages + s * SSTAGE, stages + s * SSTAGE + Op::SA, tile_of(g), g % nkb, tid);
            cp_commit();
            if (g >= kLag) {
                cp_wait<kLag>();             // this thread's copies of step g - kLag are in
                afptx::fence_proxy_async();  // ... and visible to the tensor cores
                afptx::mbar_arrive(full0 + 8 * ((g - kLag) % NS));
            }
        }
        cp_wait<0>();
        afptx::fence_proxy_async();
        for (int h = g - kLag < 0 ? 0 : g - kLag; h < g; h++) afptx::mbar_arrive(full0 + 8 * (h % NS));
    } else if (warp == 4) {
        // ---------------- MMA issuer
        for (int g = 0; g < G; g++) {
            const int s = g % NS, kb = g % nkb, i = g / nkb, b = i % NACC;
            const uint32_t acc = tmem + (uint32_t)(b * Op::NCOL);
            bool ok = true;
            if (kb == 0 && i >= NACC)  // the epilogue has read this accumulator's previous tile
                ok = wait_or_abort(tempty0 + 8 * b, (uint32_t)((i - NACC) / NACC) & 1u, abort);
            ok = ok && wait_or_abort(full0 + 8 * s, (uint32_t)(g / NS) & 1u, abort);
            if (!__all_sync(0xffffffffu, ok)) break;
            afumma::fence_after_sync();
            if (lane == 0) {
                op.mma(afptx::smem_addr(stages + s * SSTAGE), afptx::smem_addr(stages + s * SSTAGE + Op::SA),
                       afptx::smem_addr(smem), kb, acc);
                afumma::commit(empty0 + 8 * s);
                if (kb == nkb - 1) afumma::commit(tfull0 + 8 * b);
            }
            __syncwarp();
        }
        // every stage's release has arrived before the block's shared memory goes away
        for (int g = G - NS < 0 ? 0 : G - NS; g < G && !*abort; g++)
            wait_or_abort(empty0 + 8 * (g % NS), (uint32_t)(g / NS) & 1u, abort);
    } else {
        // ---------------- epilogue
        const int quarter = warp & 3;
        for (int i = 0; i < mytiles; i++) {
            const int b = i % NACC;
            if (!wait_or_abort(tfull0 + 8 * b, (uint32_t)(i / NACC) & 1u, abort)) break;
            afumma::fence_after_sync();
            op.epilogue((int)blockIdx.x + i * (int)gridDim.x, tmem + (uint32_t)(b * Op::NCOL), quarter, lane);
            afumma::fence_before_sync();
            afptx::mbar_arrive(tempty0 + 8 * b);
        }
    }
    __syncthreads();
    if (tid == 0 && *abort) atomicExch(args.err, 1);
    afumma::fence_after_sync();
    if (warp == 4) afumma::tmem_dealloc(tmem, TCOLS);
}

// One MMA step of K = 16 per pair of k groups: A and B descriptors advance by
// two K-direction core-matrix strides.
__device__ __forceinline__ void mma_k16(uint32_t tmem, uint32_t a, uint32_t lbo_a, uint32_t b, uint32_t lbo_b,
                                        uint32_t idesc, uint32_t acc)
{
    afumma::mma_bf16(tmem, afumma::smem_desc(a, lbo_a, 128), afumma::smem_desc(b, lbo_b, 128), idesc, acc);
}

// ------------------------------------------------------------ conv forward
// Rows of a tile: 32 pooling windows x 4 pixels; row r = 4 j + q is pixel q
// (raster order dy * 2 + dx) of window j, so a window's pixels sit in four
// adjacent lanes of one warp and the 2x2 max pool is two lane shuffles.
template <int CIN, int COUT>
struct FwdOp {
    static_assert(CIN == 2 || CIN % 8 == 0, "input channels: 2 or a multiple of 8");
    static_assert(COUT % 16 == 0 && COUT <= 256, "output channels");
    static constexpr int KP = (9 * CIN + 31) / 32 * 32;
    static constexpr int NS = 6, LAG = 3, NACC = 2, NCOL = COUT;
    static constexpr uint32_t SA = 128 * 32 * 2, SB = 0, RB = COUT * KP * 2;
    struct Args {
        const __nv_bfloat16* x;   // [n][H][W][CIN]
        const __nv_bfloat16* wp;  // [COUT][KP], zero for k >= 9 CIN
        const float* bias;        // [COUT]
        __nv_bfloat16* out;       // [n][H/2][W/2][COUT]
        uint8_t* idx;             // [n][H/2][W/2][COUT]: argmax | 4 if the maximum > 0 (nullable)
        int n, H, W;
        int* err;
    };
    const Args a;
    int Ho, Wo, npool;
    __device__ FwdOp(const Args& a_) : a(a_), Ho(a_.H / 2), Wo(a_.W / 2), npool(a_.n * (a_.H / 2) * (a_.W / 2)) {}
    __device__ int ntiles() const { return (npool + 31) / 32; }
    __device__ int nkb() const { return KP / 32; }
    __device__ void resident(uint8_t* res, int tid) const
    {
        const uint32_t base = afptx::smem_addr(res);
        for (int e = tid; e < COUT * KP / 8; e += kProd) {
            const int o = e / (KP / 8), kg = e % (KP / 8);
            cp16(base + kmaj_off(o, kg, COUT), a.wp + o * KP + 8 * kg, 16);
        }
    }
    // Row `tid` of a tile: its pixel's centre element and the 3x3 taps that lie
    // inside the image (bit t = dy * 3 + dx), none for rows past the end.
    __device__ const __nv_bfloat16* pixel(int tile, int tid, uint32_t& taps) const
    {
        const int pp = tile * 32 + (tid >> 2), q = tid & 3;
        taps = 0u;
        if (pp >= npool) return a.x;
        const int img = pp / (Ho * Wo), rem = pp - img * Ho * Wo;
        const int y = 2 * (rem / Wo) + (q >> 1), x = 2 * (rem % Wo) + (q & 1);
        const uint32_t rows = (y > 0 ? 1u : 0u) | 2u | (y + 1 < a.H ? 4u : 0u);
        const uint32_t cols = (x > 0 ? 1u : 0u) | 2u | (x + 1 < a.W ? 4u : 0u);
#pragma unroll
        for (int t = 0; t < 9; t++) taps |= ((rows >> (t / 3)) & (cols >> (t % 3)) & 1u) << t;
        return a.x + (((int64_t)img * a.H + y) * a.W + x) * CIN;
    }
    __device__ void stage(uint8_t* sa, uint8_t*, int tile, int kb_rt, int tid) const
    {
        const int kb = KP == 32 ? 0 : kb_rt;  // one K block: taps known at compile time
        uint32_t taps;
        const __nv_bfloat16* ctr = pixel(tile, tid, taps);
        const uint32_t base = afptx::smem_addr(sa);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int k0 = kb * 32 + 8 * c;
            const uint32_t dst = base + kmaj_off(tid, c, 128);
            if constexpr (CIN == 2) {
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int t = (k0 >> 1) + i;
                    const bool in = t < 9 && ((taps >> t) & 1u);
                    const __nv_bfloat16* src = in ? ctr + ((t / 3 - 1) * a.W + (t % 3 - 1)) * 2 : a.x;
                    cp4(dst + 4 * i, src, in ? 4u : 0u);
                }
            } else {
                const int t = k0 / CIN, i0 = k0 % CIN;
                const bool in = t < 9 && ((taps >> t) & 1u);
                const __nv_bfloat16* src = in ? ctr + ((t / 3 - 1) * a.W + (t % 3 - 1)) * CIN + i0 : a.x;
                cp16(dst, src, in ? 16u : 0u);
            }
        }
    }
    __device__ void mma(uint32_t sa, uint32_t, uint32_t res, int kb, uint32_t tmem) const
    {
        constexpr uint32_t idesc = afumma::idesc_bf16(128, COUT, 0, 0);
        constexpr uint32_t lbo_a = 16 * 128, lbo_b = COUT / 8 * 128;
#pragma unroll
        for (int j = 0; j < 2; j++)
            mma_k16(tmem, sa + 2 * j * lbo_a, lbo_a, res + (4 * kb + 2 * j) * lbo_b, lbo_b, idesc, (kb | j) != 0);
    }
    __device__ void epilogue(int tile, uint32_t tmem, int warp, int lane) const
    {
        const int tid = 32 * warp + lane, q = tid & 3;
        const int pp = tile * 32 + (tid >> 2);
#pragma unroll 1
        for (int c0 = 0; c0 < COUT; c0 += 16) {
            uint32_t v[16];
            afumma::ld_32x32b_x16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            afumma::wait_ld();
            float m[16];
            const float4* bv = reinterpret_cast<const float4*>(a.bias + c0);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float4 b4 = __ldg(bv + k);
                m[4 * k] = fmaxf(__uint_as_float(v[4 * k]) + b4.x, 0.f);
                m[4 * k + 1] = fmaxf(__uint_as_float(v[4 * k + 1]) + b4.y, 0.f);
                m[4 * k + 2] = fmaxf(__uint_as_float(v[4 * k + 2]) + b4.z, 0.f);
                m[4 * k + 3] = fmaxf(__uint_as_float(v[4 * k + 3]) + b4.w, 0.f);
            }
            int qi[16];
            if (a.idx) {  // training: the argmax travels with the maximum
#pragma unroll
                for (int i = 0; i < 16; i++) qi[i] = q;
#pragma unroll
                for (int sh = 1; sh <= 2; sh <<= 1) {
#pragma unroll
                    for (int i = 0; i < 16; i++) {
                        const float om = __shfl_xor_sync(0xffffffffu, m[i], sh);
                        const int oq = __shfl_xor_sync(0xffffffffu, qi[i], sh);
                        if (om > m[i] || (om == m[i] && oq < qi[i])) {  // the first maximum in raster order
                            m[i] = om;
                            qi[i] = oq;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int sh = 1; sh <= 2; sh <<= 1) {
#pragma unroll
                    for (int i = 0; i < 16; i++) m[i] = fmaxf(m[i], __shfl_xor_sync(0xffffffffu, m[i], sh));
                }
            }
            if (q == 0 && pp < npool) {
                uint4 o0, o1;
                o0.x = pack_bf16(m[0], m[1]);
                o0.y = pack_bf16(m[2], m[3]);
                o0.z = pack_bf16(m[4], m[5]);
                o0.w = pack_bf16(m[6], m[7]);
                o1.x = pack_bf16(m[8], m[9]);
                o1.y = pack_bf16(m[10], m[11]);
                o1.z = pack_bf16(m[12], m[13]);
                o1.w = pack_bf16(m[14], m[15]);
                uint4* dst = reinterpret_cast<uint4*>(a.out + (int64_t)pp * COUT + c0);
                dst[0] = o0;
                dst[1] = o1;
                if (a.idx) {
                    uint32_t w[4];
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        w[k] = 0;
#pragma unroll
                        for (int b = 0; b < 4; b++)
                            w[k] |= (uint32_t)(qi[4 * k + b] | (m[4 * k + b] > 0.f ? 4 : 0)) << (8 * b);
                    }
                    *reinterpret_cast<uint4*>(a.idx + (int64_t)pp * COUT + c0) = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
        }
    }
};

// ------------------------------------------------------------ data gradient
// dX (CIN channels) of a layer whose output gradient dZ has COUT channels:
// row p of a tile is pixel p; k = t * COUT + o gathers dZ at p - (tap offset).
template <int CIN, int COUT>
struct DgradOp {
    static_assert(CIN % 16 == 0 && CIN <= 256 && COUT % 8 == 0 && (9 * COUT) % 32 == 0, "channels");
    static constexpr int K = 9 * COUT;
    static constexpr int NS = 6, LAG = 3, NACC = 2, NCOL = CIN;
    static constexpr uint32_t SA = 128 * 32 * 2, SB = 0, RB = CIN * K * 2;
    struct Args {
        const __nv_bfloat16* dz;  // [n][H][W][COUT]
        const __nv_bfloat16* wd;  // [CIN][9 COUT]: W[o][t][i] at (i, t * COUT + o)
        __nv_bfloat16* dx;        // [n][H][W][CIN]
        int n, H, W;
        int* err;
    };
    const Args a;
    int P;
    __device__ DgradOp(const Args& a_) : a(a_), P(a_.n * a_.H * a_.W) {}
    __device__ int ntiles() const { return (P + 127) / 128; }
    __device__ int nkb() const { return K / 32; }
    __device__ void resident(uint8_t* res, int tid) const
    {
        const uint32_t base = afptx::smem_addr(res);
        for (int e = tid; e < CIN * K / 8; e += kProd) {
            const int i = e / (K / 8), kg = e % (K / 8);
            cp16(base + kmaj_off(i, kg, CIN), a.wd + i * K + 8 * kg, 16);
        }
    }
    __device__ void stage(uint8_t* sa, uint8_t*, int tile, int kb, int tid) const
    {
        // tap t = dy * 3 + dx reads dZ at (y + 1 - dy, x + 1 - dx): bit t set when inside
        const int p = tile * 128 + tid;
        uint32_t taps = 0u;
        const __nv_bfloat16* ctr = a.dz;
        if (p < P) {
            const int img = p / (a.H * a.W), rem = p - img * a.H * a.W, y = rem / a.W, x = rem % a.W;
            const uint32_t rows = (y + 1 < a.H ? 1u : 0u) | 2u | (y > 0 ? 4u : 0u);
            const uint32_t cols = (x + 1 < a.W ? 1u : 0u) | 2u | (x > 0 ? 4u : 0u);
#pragma unroll
            for (int t = 0; t < 9; t++) taps |= ((rows >> (t / 3)) & (cols >> (t % 3)) & 1u) << t;
            ctr = a.dz + (int64_t)p * COUT;
        }
        const uint32_t base = afptx::smem_addr(sa);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int k0 = kb * 32 + 8 * c, t = k0 / COUT, o0 = k0 % COUT;
            const bool in = (taps >> t) & 1u;
            const __nv_bfloat16* src = in ? ctr + ((1 - t / 3) * a.W + (1 - t % 3)) * COUT + o0 : a.dz;
            cp16(base + kmaj_off(tid, c, 128), src, in ? 16u : 0u);
        }
    }
    __device__ void mma(uint32_t sa, uint32_t, uint32_t res, int kb, uint32_t tmem) const
    {
        constexpr uint32_t idesc = afumma::idesc_bf16(128, CIN, 0, 0);
        constexpr uint32_t lbo_a = 16 * 128, lbo_b = CIN / 8 * 128;
#pragma unroll
        for (int j = 0; j < 2; j++)
            mma_k16(tmem, sa + 2 * j * lbo_a, lbo_a, res + (4 * kb + 2 * j) * lbo_b, lbo_b, idesc, (kb | j) != 0);
    }
    __device__ void epilogue(int tile, uint32_t tmem, int warp, int lane) const
    {
        const int p = tile * 128 + 32 * warp + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < CIN; c0 += 16) {
            uint32_t v[16];
            afumma::ld_32x32b_x16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            afumma::wait_ld();
            if (p < P) {
                uint4 o0, o1;
                o0.x = pack_bf16(__uint_as_float(v[0]), __uint_as_float(v[1]));
                o0.y = pack_bf16(__uint_as_float(v[2]), __uint_as_float(v[3]));
                o0.z = pack_bf16(__uint_as_float(v[4]), __uint_as_float(v[5]));
                o0.w = pack_bf16(__uint_as_float(v[6]), __uint_as_float(v[7]));
                o1.x = pack_bf16(__uint_as_float(v[8]), __uint_as_float(v[9]));
                o1.y = pack_bf16(__uint_as_float(v[10]), __uint_as_float(v[11]));
                o1.z = pack_bf16(__uint_as_float(v[12]), __uint_as_float(v[13]));
                o1.w = pack_bf16(__uint_as_float(v[14]), __uint_as_float(v[15]));
                uint4* dst = reinterpret_cast<uint4*>(a.dx + (int64_t)p * CIN + c0);
                dst[0] = o0;
                dst[1] = o1;
            }
        }
    }
};

// ------------------------------------------------------------ weight gradient
// Tile = a run of `kchunk` pixels (K, split across the grid); stages of BKW
// pixels.  A = dZ^T and B = the gathered input (rows n = t * CIN + i), both
// MN-major: a 16-byte chunk is 8 channels of one pixel.  A holds only the
// COUT real rows (K-direction stride COUT/8 core matrices); the MMA's other
// rows (M = 128) read whatever follows in the stage, and their results are
// never read.  Partial sums go to the fp32 gradient with atomics.
template <int CIN, int COUT, int BKW>
struct WgradOp {
    static_assert((CIN == 2 || CIN % 8 == 0) && COUT % 16 == 0 && COUT <= 128 && BKW % 64 == 0, "shapes");
    static constexpr int K9 = 9 * CIN, NP = (K9 + 15) / 16 * 16;
    static_assert(NP <= 256 || (NP % 32 == 0 && NP <= 512), "columns");
    static constexpr int NS = 4, LAG = 3, NACC = 1, NCOL = NP;
    static constexpr uint32_t SA = COUT * BKW * 2, SB = NP * BKW * 2, RB = 0;
    static_assert(SB >= 16 * 128, "the padding rows of A must read inside the stage");
    struct Args {
        const __nv_bfloat16* dz;  // [n][H][W][COUT]
        const __nv_bfloat16* x;   // [n][H][W][CIN]
        float* grad;              // [COUT][9 CIN], accumulated
        int n, H, W, kchunk;      // kchunk: pixels per tile, a multiple of BKW
        int* err;
    };
    const Args a;
    int P;
    __device__ WgradOp(const Args& a_) : a(a_), P(a_.n * a_.H * a_.W) {}
    __device__ int ntiles() const { return (P + a.kchunk - 1) / a.kchunk; }
    __device__ int nkb() const { return a.kchunk / BKW; }
    __device__ void resident(uint8_t*, int) const {}
    __device__ void stage(uint8_t* sa, uint8_t* sb, int tile, int kb, int tid) const
    {
        const uint32_t ba = afptx::smem_addr(sa), bb = afptx::smem_addr(sb);
#pragma unroll 1
        for (int r = 0; r < BKW / 64; r++) {
            // every chunk of this thread in this pass is pixel k of the stage
            const int k = 64 * r + (tid & 63), p = tile * a.kchunk + kb * BKW + k;
            uint32_t taps = 0u;  // bit t = dy * 3 + dx: tap (y + dy - 1, x + dx - 1) inside the image
            const __nv_bfloat16* ctr = a.x;
            const bool valid = p < P;
            if (valid) {
                const int img = p / (a.H * a.W), rem = p - img * a.H * a.W, y = rem / a.W, x = rem % a.W;
                const uint32_t rows = (y > 0 ? 1u : 0u) | 2u | (y + 1 < a.H ? 4u : 0u);
                const uint32_t cols = (x > 0 ? 1u : 0u) | 2u | (x + 1 < a.W ? 4u : 0u);
#pragma unroll
                for (int t = 0; t < 9; t++) taps |= ((rows >> (t / 3)) & (cols >> (t % 3)) & 1u) << t;
                ctr = a.x + (int64_t)p * CIN;
            }
            for (int g = tid >> 6; g < COUT / 8; g += 2)
                cp16(ba + mnmaj_off(g, k, COUT), valid ? a.dz + (int64_t)p * COUT + 8 * g : a.dz, valid ? 16u : 0u);
            for (int g = tid >> 6; g < NP / 8; g += 2) {
                const uint32_t dst = bb + mnmaj_off(g, k, NP);
                if constexpr (CIN == 2) {
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const int t = 4 * g + i;
                        const bool in = t < 9 && ((taps >> t) & 1u);
                        cp4(dst + 4 * i, in ? ctr + ((t / 3 - 1) * a.W + (t % 3 - 1)) * 2 : a.x, in ? 4u : 0u);
                    }
                } else {
                    const int n0 = 8 * g, t = n0 / CIN, i0 = n0 % CIN;
                    const bool in = t < 9 && ((taps >> t) & 1u);
                    cp16(dst, in ? ctr + ((t / 3 - 1) * a.W + (t % 3 - 1)) * CIN + i0 : a.x, in ? 16u : 0u);
                }
            }
        }
    }
    __device__ void mma(uint32_t sa, uint32_t sb, uint32_t, int kb, uint32_t tmem) const
    {
        constexpr uint32_t lbo_a = COUT / 8 * 128, lbo_b = NP / 8 * 128;
#pragma unroll
        for (int j = 0; j < BKW / 16; j++) {
            const uint32_t acc = (kb | j) != 0;
            if constexpr (NP <= 256) {
                mma_k16(tmem, sa + 2 * j * lbo_a, lbo_a, sb + 2 * j * lbo_b, lbo_b, afumma::idesc_bf16(128, NP, 1, 1),
                        acc);
            } else {  // two MMAs of NP / 2 columns each
                constexpr uint32_t idesc = afumma::idesc_bf16(128, NP / 2, 1, 1);
                mma_k16(tmem, sa + 2 * j * lbo_a, lbo_a, sb + 2 * j * lbo_b, lbo_b, idesc, acc);
                mma_k16(tmem + NP / 2, sa + 2 * j * lbo_a, lbo_a, sb + 2 * j * lbo_b + (NP / 16) * 128, lbo_b, idesc,
                        acc);
            }
        }
    }
    __device__ void epilogue(int, uint32_t tmem, int warp, int lane) const
    {
        if (32 * warp >= COUT) return;  // warp-uniform: these lanes hold padding rows only
        const int o = 32 * warp + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < NP; c0 += 16) {
            uint32_t v[16];
            afumma::ld_32x32b_x16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            afumma::wait_ld();
            if (o < COUT) {
#pragma unroll
                for (int i = 0; i < 16; i++)
                    if (c0 + i < K9) atomicAdd(a.grad + o * K9 + c0 + i, __uint_as_float(v[i]));
            }
        }
    }
};

// ------------------------------------------------------------ plain GEMM
// C[M][N] (ldc) = sum_k A[m][k] B[k][n]; A K-major ([M][lda]) or M-major
// ([K][lda]), B K-major ([N][ldb]) or N-major ([K][ldb]); tiles 128 x 64,
// K split into `kchunk` runs (atomic epilogue only).
template <bool AK, bool BK, int EPI>
struct GemmOp {
    static constexpr int NS = 4, LAG = 3, NACC = 2, NCOL = 64;
    static constexpr uint32_t SA = 128 * 32 * 2, SB = 64 * 32 * 2, RB = 0;
    struct Args {
        const __nv_bfloat16* A;
        const __nv_bfloat16* B;
        float* C;
        const float* bias;
        int lda, ldb, ldc, M, N, K, kchunk, mt, nt;
        int* err;
    };
    const Args a;
    __device__ GemmOp(const Args& a_) : a(a_) {}
    __device__ int ntiles() const { return a.mt * a.nt * ((a.K + a.kchunk - 1) / a.kchunk); }
    __device__ int nkb() const { return a.kchunk / 32; }
    __device__ void resident(uint8_t*, int) const {}
    __device__ void coords(int tile, int& m0, int& n0, int& k0) const
    {
        const int mt = tile % a.mt, rest = tile / a.mt;
        m0 = 128 * mt;
        n0 = 64 * (rest % a.nt);
        k0 = a.kchunk * (rest / a.nt);
    }
    __device__ void stage(uint8_t* sa, uint8_t* sb, int tile, int kb, int tid) const
    {
        int m0, n0, k0;
        coords(tile, m0, n0, k0);
        k0 += 32 * kb;
        const int kend = min(a.K, k0 - 32 * kb + a.kchunk);
        const uint32_t ba = afptx::smem_addr(sa), bb = afptx::smem_addr(sb);
        if constexpr (AK) {
            const int m = m0 + tid;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int k = k0 + 8 * c;
                const bool in = m < a.M && k < kend;
                cp16(ba + kmaj_off(tid, c, 128), in ? a.A + (int64_t)m * a.lda + k : a.A, in ? 16u : 0u);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int e = tid + kProd * i, mg = e & 15, k = e >> 4, m = m0 + 8 * mg;
                const bool in = m < a.M && k0 + k < kend;
                const uint32_t bytes = in ? (uint32_t)min(16, 2 * (a.M - m)) : 0u;
                cp16(ba + mnmaj_off(mg, k, 128), in ? a.A + (int64_t)(k0 + k) * a.lda + m : a.A, bytes);
            }
        }
        if constexpr (BK) {
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int e = tid + kProd * i, r = e >> 2, c = e & 3, n = n0 + r, k = k0 + 8 * c;
                const bool in = n < a.N && k < kend;
                cp16(bb + kmaj_off(r, c, 64), in ? a.B + (int64_t)n * a.ldb + k : a.B, in ? 16u : 0u);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int e = tid + kProd * i, ng = e & 7, k = e >> 3, n = n0 + 8 * ng;
                const bool in = n < a.N && k0 + k < kend;
                const uint32_t bytes = in ? (uint32_t)min(16, 2 * (a.N - n)) : 0u;
                cp16(bb + mnmaj_off(ng, k, 64), in ? a.B + (int64_t)(k0 + k) * a.ldb + n : a.B, bytes);
            }
        }
    }
    __device__ void mma(uint32_t sa, uint32_t sb, uint32_t, int kb, uint32_t tmem) const
    {
        constexpr uint32_t idesc = afumma::idesc_bf16(128, 64, AK ? 0 : 1, BK ? 0 : 1);
        constexpr uint32_t lbo_a = 16 * 128, lbo_b = 8 * 128;
#pragma unroll
        for (int j = 0; j < 2; j++)
            mma_k16(tmem, sa + 2 * j * lbo_a, lbo_a, sb + 2 * j * lbo_b, lbo_b, idesc, (kb | j) != 0);
    }
    __device__ void epilogue(int tile, uint32_t tmem, int warp, int lane) const
    {
        int m0, n0, k0;
        coords(tile, m0, n0, k0);
        const int m = m0 + 32 * warp + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < 64; c0 += 16) {
            uint32_t v[16];
            afumma::ld_32x32b_x16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            afumma::wait_ld();
            if (m < a.M) {
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const int n = n0 + c0 + i;
                    if (n >= a.N) continue;
                    float* c = a.C + (int64_t)m * a.ldc + n;
                    const float x = __uint_as_float(v[i]);
                    if constexpr (EPI == NN_EPI_STORE) *c = x;
                    else if constexpr (EPI == NN_EPI_BIAS_RELU) *c = fmaxf(x + __ldg(a.bias + n), 0.f);
                    else atomicAdd(c, x);
                }
            }
        }
    }
};

// Wd[i][t * COUT + o] = bf16(W[o][t][i]) (the data gradient's resident operand)
__global__ void k_pack_wd(const float* __restrict__ w, int cin, int cout, __nv_bfloat16* __restrict__ wd)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cin * 9 * cout) return;
    const int i = e / (9 * cout), r = e % (9 * cout), t = r / cout, o = r % cout;
    wd[e] = __float2bfloat16(w[(o * 9 + t) * cin + i]);
}

// Resident blocks per device for Op (computed once per device, under a lock:
// model calls may come from several host threads).
template <class Op>
int resident_blocks(int dev, size_t smem, int* out)
{
    static std::mutex mu;
    static std::map<int, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) {
        *out = it->second;
        return AF_OK;
    }
    AF_CUDA(cudaFuncSetAttribute(k_umma<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    AF_CUDA(cudaFuncSetAttribute(k_umma<Op>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    int nsm = 0, smem_sm = 0, per_sm = 0;
    AF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    AF_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    AF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_umma<Op>, kBlock, smem));
    // resident blocks: by shared memory (1 KB reserved per block), warps, and
    // the 512 tensor-memory columns each block takes its share of
    const int by_smem = smem_sm / (int)(smem + 1024 + 256);
    int b = by_smem < 64 / (kBlock / 32) ? by_smem : 64 / (kBlock / 32);
    if (per_sm > b) b = per_sm;
    const int by_tmem = 512 / pow2_cols(Op::NACC * Op::NCOL);
    if (b > by_tmem) b = by_tmem;
    *out = cache[dev] = (b < 1 ? 1 : b) * nsm;
    return AF_OK;
}

template <class Op>
int launch(const typename Op::Args& a, int ntiles, cudaStream_t s, const char* what)
{
    if (ntiles <= 0) return AF_OK;
    const size_t smem = Op::RB + (size_t)Op::NS * (Op::SA + Op::SB);
    int dev = 0, blocks = 0;
    AF_CUDA(cudaGetDevice(&dev));
    if (int rc = resident_blocks<Op>(dev, smem, &blocks)) return rc;
    const int grid = ntiles < blocks ? ntiles : blocks;
    k_umma<Op><<<grid, kBlock, smem, s>>>(a);
    return af_cuda_check(cudaGetLastError(), what);
}

int sm_count()
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm > 0 ? nsm : 1;
}

}  // namespace

int nn_conv_fwd(int layer, const __nv_bfloat16* x, int n, int H, int W, const __nv_bfloat16* wp, const float* bias,
                __nv_bfloat16* out, uint8_t* idx, int* err, cudaStream_t s)
{
    const int tiles = (n * (H / 2) * (W / 2) + 31) / 32;
#define AF_FWD(L, CI, CO)                                                                        \
    if (layer == L) {                                                                            \
        typename FwdOp<CI, CO>::Args a{x, wp, bias, out, idx, n, H, W, err};                     \
        return launch<FwdOp<CI, CO>>(a, tiles, s, "conv forward (tcgen05)");                     \
    }
    AF_FWD(0, 2, 16)
    AF_FWD(1, 16, 32)
    AF_FWD(2, 32, 64)
#undef AF_FWD
    return af_set_error(AF_EINVAL, "conv forward: layer %d", layer);
}

int nn_conv_dgrad(int layer, const __nv_bfloat16* dz, int n, int H, int W, const __nv_bfloat16* wd,
                  __nv_bfloat16* dx, int* err, cudaStream_t s)
{
    const int tiles = (n * H * W + 127) / 128;
#define AF_DG(L, CI, CO)                                                             \
    if (layer == L) {                                                                \
        typename DgradOp<CI, CO>::Args a{dz, wd, dx, n, H, W, err};                  \
        return launch<DgradOp<CI, CO>>(a, tiles, s, "conv data gradient (tcgen05)"); \
    }
    AF_DG(1, 16, 32)
    AF_DG(2, 32, 64)
#undef AF_DG
    return af_set_error(AF_EINVAL, "conv data gradient: layer %d", layer);
}

int nn_conv_wgrad(int layer, const __nv_bfloat16* dz, const __nv_bfloat16* x, int n, int H, int W, float* grad,
                  int* err, cudaStream_t s)
{
    // about two tiles of pixels per SM, each a multiple of 256 pixels
    const int64_t P = (int64_t)n * H * W;
    int64_t kc = (P + 2 * sm_count() - 1) / (2 * sm_count());
    kc = (kc + 255) / 256 * 256;
    const int tiles = (int)((P + kc - 1) / kc);
#define AF_WG(L, CI, CO, BKW)                                                                      \
    if (layer == L) {                                                                              \
        typename WgradOp<CI, CO, BKW>::Args a{dz, x, grad, n, H, W, (int)kc, err};                 \
        return launch<WgradOp<CI, CO, BKW>>(a, tiles, s, "conv weight gradient (tcgen05)");        \
    }
    AF_WG(0, 2, 16, 256)
    AF_WG(1, 16, 32, 128)
    AF_WG(2, 32, 64, 64)
#undef AF_WG
    return af_set_error(AF_EINVAL, "conv weight gradient: layer %d", layer);
}

int nn_pack_wd(const float* w, int cin, int cout, __nv_bfloat16* wd, cudaStream_t s)
{
    k_pack_wd<<<(cin * 9 * cout + 255) / 256, 256, 0, s>>>(w, cin, cout, wd);
    return af_cuda_check(cudaGetLastError(), "pack data-gradient weights");
}

int nn_gemm(int layout, int epi, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
            int splits, float* C, int ldc, const float* bias, int* err, cudaStream_t s)
{
    if ((lda & 7) || (ldb & 7) || (K & 7) || ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || M < 1 || N < 1 || K < 1 ||
        splits < 1)
        return af_set_error(AF_EINVAL,
                            "gemm: K and the leading dimensions must be multiples of 8, operands 16-byte aligned");
    if (epi != NN_EPI_ATOMIC) splits = 1;
    int kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + 31) / 32 * 32;
    const int mt = (M + 127) / 128, nt = (N + 63) / 64, tiles = mt * nt * ((K + kchunk - 1) / kchunk);
#define AF_GEMM_EPI(AKv, BKv, E)                                                          \
    {                                                                                     \
        typename GemmOp<AKv, BKv, E>::Args a{A, B, C, bias, lda, ldb, ldc, M, N, K, kchunk, mt, nt, err}; \
        return launch<GemmOp<AKv, BKv, E>>(a, tiles, s, "gemm (tcgen05)");               \
    }
#define AF_GEMM_CASE(L, AKv, BKv)                                     \
    case L:                                                           \
        if (epi == NN_EPI_STORE) AF_GEMM_EPI(AKv, BKv, NN_EPI_STORE)  \
        if (epi == NN_EPI_BIAS_RELU) AF_GEMM_EPI(AKv, BKv, NN_EPI_BIAS_RELU) \
        AF_GEMM_EPI(AKv, BKv, NN_EPI_ATOMIC)
    switch (layout) {
        AF_GEMM_CASE(NN_A_K_B_K, true, true)
        AF_GEMM_CASE(NN_A_K_B_N, true, false)
        AF_GEMM_CASE(NN_A_M_B_N, false, false)
        AF_GEMM_CASE(NN_A_M_B_K, false, true)
    }
#undef AF_GEMM_CASE
#undef AF_GEMM_EPI
    return af_set_error(AF_EINVAL, "gemm: unknown layout");
}
