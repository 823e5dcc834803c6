// umma.cuh -- inline-PTX helpers for the 5th-generation tensor cores
// (tcgen05): tensor-memory allocation, shared-memory matrix descriptors,
// the instruction descriptor of kind::f16 (bf16 operands, fp32 accumulate),
// the MMA itself, its completion commit onto an mbarrier, and tensor-memory
// loads for the epilogue.  cta_group::1 throughout (one SM per tile).
//
// Operand tiles sit in shared memory in the no-swizzle canonical layout:
// "core matrices" of 8 rows x 16 bytes (8 bf16), each 128 contiguous bytes.
// A K-major operand's core matrix holds 8 rows (M or N) x 8 consecutive K;
// an MN-major operand's holds 8 consecutive K rows x 8 consecutive M (or N)
// elements.  The descriptor gives the byte distance between core matrices
// adjacent along K (the leading-dimension offset) and along M / N (the
// stride-dimension offset).
#pragma once
#include <stdint.h>

namespace afumma {

// Tensor memory: one warp allocates `ncols` columns (a power of two, 32..512)
// of all 128 lanes and writes the base address to shared memory at `slot`.
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle: start address, leading-
// dimension (K) and stride-dimension (M / N) byte offsets between core
// matrices; bits 46-47 hold the descriptor version (1 on this architecture).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of tcgen05.mma kind::f16: D fp32, A and B bf16,
// A / B K-major (0) or MN-major (1), shape M x N (M = 64 or 128; N a
// multiple of 16 up to 256 for M = 128).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (tensor memory) = A x B^T (+ D when `accumulate`); issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The mbarrier at `bar` receives one arrival once every tcgen05 operation
// this thread issued before has completed.
__device__ __forceinline__ void commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns: thread i of the warp gets lane
// (taddr's lane + i), columns taddr's column .. + 15.
__device__ __forceinline__ void ld_32x32b_x16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One non-blocking test of an mbarrier phase (never suspends the thread).
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for a phase by spinning on test_wait (a pipeline hand-off is a few
// hundred cycles; a suspended try_wait can return much later than the phase
// completes), giving up after kWaitNs of wall time or when another thread
// gave up; a wait that gives up raises the block's abort flag.  backoff_ns > 0
// sleeps that long between polls after the first few (for warps whose
// latency matters less than the issue slots they would take from others).
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort,
                                              uint32_t backoff_ns = 0)
{
    if (mbar_test_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t i = 1;; i++) {
        if (mbar_test_wait(bar, parity)) return true;
        if (backoff_ns && i > 4) __nanosleep(backoff_ns);
        if ((i & 255) == 0) {
            if (*abort) return false;
            if (globaltimer_ns() - t0 > kWaitNs) break;
        }
    }
    *abort = 1;
    return false;
}

}  // namespace afumma
