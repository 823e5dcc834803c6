// conv_umma.cu -- a plain GEMM on the 5th-generation tensor cores
// (tcgen05.mma kind::f16: bf16 operands, fp32 accumulators in tensor
// memory), C = A B in the four operand layouts (af_nn_gemm), with a stored,
// bias + ReLU or split-K atomic epilogue.  The classifier's convolutions have
// their own TMA-fed kernel (conv_tma.cu).
//
// 128 producer threads stage operand tiles with 16-byte cp.async copies
// through L1, zero filled outside the matrix, straight into the no-swizzle
// canonical layout of umma.cuh; thread 0 of the MMA warp issues a stage's
// MMAs and commits them onto the stage's mbarrier, which frees the stage for
// the copies; after a tile's last stage every epilogue warp reads its 32
// tensor-memory lanes (rows) back with tcgen05.ld.  Every mbarrier wait is
// bounded: a wait that runs out raises the caller's error flag and the kernel
// leaves cleanly.
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

// cp.async of 16 bytes through L1; `bytes` < 16 zero-fills the rest (0: no read)
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
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
            if (g >= NS && !afumma::wait_or_abort(empty0 + 8 * s, (uint32_t)(g / NS - 1) & 1u, abort)) break;
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
                ok = afumma::wait_or_abort(tempty0 + 8 * b, (uint32_t)((i - NACC) / NACC) & 1u, abort);
            ok = ok && afumma::wait_or_abort(full0 + 8 * s, (uint32_t)(g / NS) & 1u, abort);
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
            afumma::wait_or_abort(empty0 + 8 * (g % NS), (uint32_t)(g / NS) & 1u, abort);
    } else {
        // ---------------- epilogue
        const int quarter = warp & 3;
        for (int i = 0; i < mytiles; i++) {
            const int b = i % NACC;
            if (!afumma::wait_or_abort(tfull0 + 8 * b, (uint32_t)(i / NACC) & 1u, abort)) break;
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

}  // namespace

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
