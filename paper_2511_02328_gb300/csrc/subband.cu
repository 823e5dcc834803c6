// subband.cu -- two-stage subband dedispersion (Sec. 2.3, Eqs. stage1,
// residual, stage2) for plans made by af_plan_subband.
//
//   stage 1  I(j,s,u) = sum_{c in s} X[c][u + D[j][c]]      (coarse DM j, subband s)
//   stage 2  Y[m][v]  = sum_s I(j(m), s, v + R[m][s])        (fine DM m, j(m) = m / n0)
//
// The time axis is processed in blocks of L outputs (the paper's blocking,
// Eq. L1): for outputs [v0, v0 + L) stage 1 fills I for u in [v0, v0 + L + Rmax)
// into the plan's scratch, then stage 2 reads it.  Both stages are exact
// integer sums, so the plane equals the brute-force sum with the effective
// delays D[j(m)][c] + R[m][s(c)].
//
// Stage 1 is the tile kernel of tile.cuh in subband mode: rows = coarse DMs
// (11 per block), channels streamed subband by subband, one scratch row
// stored per (row, subband).  Its table delays are staggered per (row,
// subband) so that a block's delay spread is the within-subband dispersion
// only (see tile.cuh).
//
// Stage 2 (k_sb_stage2): one block per (coarse DM, time tile of TV outputs);
// SC scratch rows at a time are brought into shared memory by bulk
// asynchronous copies (double-buffered, mbarrier completion); each thread owns
// P outputs of every fine DM of the group and adds the subbands' shifted
// values from shared memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "ptx.cuh"
#include "tile.cuh"

namespace {

constexpr int kSbNW = 11;  // stage-1 block shape (rows x 128-output groups)
constexpr int kSbM = 8;
constexpr int kS2Threads = 256;
constexpr int kS2BufBytes = 24576;       // target bytes per stage-2 buffer
constexpr int64_t kScratchBudget = (int64_t)1 << 30;  // default stage-1 scratch
constexpr int64_t kMaxDefaultL = (int64_t)1 << 18;
constexpr uint32_t kS2WaitLimit = afptx::kMbarWaitPolls;
constexpr int kS2RBytes = 16384;          // residual-shift table kept in shared memory up to this size

template <typename T, int NM>
__global__ void __launch_bounds__(kS2Threads)
k_sb_stage2(const T* __restrict__ I, int64_t ipitch, int nsub, int n0, int ndm, const int32_t* __restrict__ R,
            int rw, int sc, int64_t v0, int64_t lcur, int64_t nout, unsigned vtiles, int32_t* __restrict__ Y,
            af_rowstats_t* __restrict__ stats, int* err, int rsmem)
{
    constexpr int P = 64 / NM;
    constexpr int TV = kS2Threads * P;
    extern __shared__ __align__(16) uint8_t smem[];
    T* buf = reinterpret_cast<T*>(smem);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)2 * sc * rw * sizeof(T));
    int32_t* sR = reinterpret_cast<int32_t*>(bars + 2);  // [NM][nsub] residual shifts of the group
    const uint32_t bar0 = afptx::smem_addr(bars);
    const int tid = threadIdx.x;
    const int j = (int)(blockIdx.x / vtiles);
    const int64_t vl0 = (int64_t)(blockIdx.x % vtiles) * TV;
    const int m0 = j * n0;
    const int nm = min(n0, ndm - m0);
    const int nchunk = (nsub + sc - 1) / sc;
    const T* Ij = I + (int64_t)j * nsub * ipitch + vl0;

    if (tid == 0) {
        afptx::mbar_init(bar0, 1);
        afptx::mbar_init(bar0 + 8, 1);
        afptx::fence_mbar_init();
    }
    if (rsmem)
        for (int i = tid; i < nm * nsub; i += kS2Threads) sR[i] = __ldg(R + (int64_t)m0 * nsub + i);
    const int32_t* Rg = rsmem ? sR : R + (int64_t)m0 * nsub;  // shared, or global for very many subbands
    __syncthreads();

    // chunk k = subbands [k*sc, k*sc + ns) into buffer k & 1
    auto issue = [&](int k) {
        const int s0 = k * sc, ns = min(sc, nsub - s0);
        const uint32_t bytes = (uint32_t)(rw * sizeof(T));
        const uint32_t bar = bar0 + 8 * (k & 1);
        afptx::fence_proxy_async();
        afptx::mbar_arrive_expect_tx(bar, bytes * (uint32_t)ns);
        T* dst = buf + (size_t)(k & 1) * sc * rw;
        for (int i = 0; i < ns; i++)
            afptx::bulk_g2s(afptx::smem_addr(dst + (size_t)i * rw), Ij + (int64_t)(s0 + i) * ipitch, bytes, bar);
    };

    int acc[NM][P];
#pragma unroll
    for (int m = 0; m < NM; m++)
#pragma unroll
        for (int p = 0; p < P; p++) acc[m][p] = 0;

    if (tid == 0) issue(0);
    int k = 0;
    bool failed = false;
    for (; k < nchunk; k++) {
        if (tid == 0 && k + 1 < nchunk) issue(k + 1);  // its buffer was released by the barrier ending k-1
        const bool ok = afptx::mbar_wait_bounded(bar0 + 8 * (k & 1), (uint32_t)(k >> 1) & 1u, kS2WaitLimit);
        if (!__syncthreads_and(ok)) {
            failed = true;
            break;
        }
        const T* b = buf + (size_t)(k & 1) * sc * rw + tid;
        const int s0 = k * sc, ns = min(sc, nsub - s0);
        for (int i = 0; i < ns; i++) {
            const T* row = b + (size_t)i * rw;
            const int32_t* Rs = Rg + s0 + i;
#pragma unroll
            for (int m = 0; m < NM; m++) {
                if (m < nm) {
                    const int r = Rs[m * nsub];
#pragma unroll
                    for (int p = 0; p < P; p++) acc[m][p] += (int)row[r + kS2Threads * p];
                }
            }
        }
        __syncthreads();
    }
    if (failed) {
        if (tid == 0) {
            atomicExch(err, 1);
            // leave no copy in flight: chunk k and, if issued, chunk k + 1
            for (int k2 = k; k2 < min(k + 2, nchunk); k2++)
                afptx::mbar_wait_bounded(bar0 + 8 * (k2 & 1), (uint32_t)(k2 >> 1) & 1u, kS2WaitLimit);
        }
        return;
    }

    const int lane = tid & 31;
#pragma unroll
    for (int m = 0; m < NM; m++) {
        if (m < nm) {
            long long ss = 0, qq = 0;
            int32_t* y = Y + (int64_t)(m0 + m) * nout + v0;
#pragma unroll
            for (int p = 0; p < P; p++) {
                const int64_t vl = vl0 + tid + kS2Threads * p;
                if (vl < lcur) {
                    const int v = acc[m][p];
                    y[vl] = v;
                    ss += v;
                    qq += (long long)v * v;
                }
            }
            if (stats) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    ss += __shfl_xor_sync(0xffffffffu, ss, o);
                    qq += __shfl_xor_sync(0xffffffffu, qq, o);
                }
                if (lane == 0) {
                    atomicAdd(reinterpret_cast<unsigned long long*>(&stats[m0 + m].sum), (unsigned long long)ss);
                    atomicAdd(reinterpret_cast<unsigned long long*>(&stats[m0 + m].sumsq), (unsigned long long)qq);
                }
            }
        }
    }
}

template <typename T, int NM>
struct Stage2 {
    static const void* fn() { return (const void*)k_sb_stage2<T, NM>; }
    static void launch(unsigned grid, size_t smem, cudaStream_t s, const T* I, int64_t ipitch, int nsub, int n0,
                       int ndm, const int32_t* R, int rw, int sc, int64_t v0, int64_t lcur, int64_t nout,
                       unsigned vtiles, int32_t* Y, af_rowstats_t* stats, int* err)
    {
        const int rsmem = (size_t)NM * nsub * 4 <= (size_t)kS2RBytes;
        k_sb_stage2<T, NM><<<grid, kS2Threads, smem, s>>>(I, ipitch, nsub, n0, ndm, R, rw, sc, v0, lcur, nout, vtiles,
                                                          Y, stats, err, rsmem);
    }
};

int nm_class(int n0) { return n0 <= 4 ? 4 : n0 <= 8 ? 8 : n0 <= 16 ? 16 : 32; }
int tv_of(int n0) { return kS2Threads * (64 / nm_class(n0)); }

// Stage-2 shared-memory geometry: rows of rw elements, sc rows per buffer.
void s2_geometry(af_plan_t p, int* rw, int* sc, size_t* smem)
{
    const size_t es = p->sb.i16 ? 2 : 4;
    *rw = (tv_of(p->sb_n0) + p->sb_rmax + 7) & ~7;
    *sc = std::max(1, std::min(p->sb_nsub, (int)(kS2BufBytes / ((size_t)*rw * es))));
    const size_t rbytes = (size_t)nm_class(p->sb_n0) * p->sb_nsub * 4;
    *smem = 2 * (size_t)(*sc) * (size_t)(*rw) * es + 16 + (rbytes <= (size_t)kS2RBytes ? rbytes : 0);
}

template <typename T>
const void* s2_fn(int n0)
{
    switch (nm_class(n0)) {
    case 4: return Stage2<T, 4>::fn();
    case 8: return Stage2<T, 8>::fn();
    case 16: return Stage2<T, 16>::fn();
    default: return Stage2<T, 32>::fn();
    }
}

template <typename T>
void s2_launch(int n0, unsigned grid, size_t smem, cudaStream_t s, const T* I, int64_t ipitch, int nsub, int ndm,
               const int32_t* R, int rw, int sc, int64_t v0, int64_t lcur, int64_t nout, unsigned vtiles, int32_t* Y,
               af_rowstats_t* stats, int* err)
{
    switch (nm_class(n0)) {
    case 4: Stage2<T, 4>::launch(grid, smem, s, I, ipitch, nsub, n0, ndm, R, rw, sc, v0, lcur, nout, vtiles, Y, stats, err); break;
    case 8: Stage2<T, 8>::launch(grid, smem, s, I, ipitch, nsub, n0, ndm, R, rw, sc, v0, lcur, nout, vtiles, Y, stats, err); break;
    case 16: Stage2<T, 16>::launch(grid, smem, s, I, ipitch, nsub, n0, ndm, R, rw, sc, v0, lcur, nout, vtiles, Y, stats, err); break;
    default: Stage2<T, 32>::launch(grid, smem, s, I, ipitch, nsub, n0, ndm, R, rw, sc, v0, lcur, nout, vtiles, Y, stats, err); break;
    }
}

}  // namespace

void af_sb_free(af_plan_t p)
{
    af_tile_tables_free(&p->sb.tile);
    cudaFree(p->sb.d_stag);
    cudaFree(p->sb.d_first);
    cudaFree(p->sb.d_r);
    cudaFree(p->sb.d_I);
    p->sb.d_stag = nullptr;
    p->sb.d_first = nullptr;
    p->sb.d_r = nullptr;
    p->sb.d_I = nullptr;
}

int af_sb_prepare(af_plan_t p)
{
    const int nchan = p->nchan, nsub = p->sb_nsub, nc = p->sb_ncoarse;
    const std::vector<int32_t>& first = p->sb_first;
    const std::vector<int32_t>& Dc = p->sb_dc;

    // top channel (highest frequency, smallest delay) of each subband
    std::vector<int> top(nsub);
    for (int s = 0; s < nsub; s++) top[s] = p->f_hi > p->f_lo ? first[s + 1] - 1 : first[s];

    // stagger per (row, subband): the row's delay at the subband's top channel
    // minus the smallest such delay in its block of kSbNW rows (padding rows
    // repeat the last coarse DM, as the tile tables do)
    const int nblk = (nc + kSbNW - 1) / kSbNW, npad = nblk * kSbNW;
    std::vector<int32_t> stag((size_t)npad * nsub), e((size_t)nc * nchan);
    int32_t maxstag = 0;
    for (int b = 0; b < nblk; b++)
        for (int s = 0; s < nsub; s++) {
            int32_t lo = INT32_MAX;
            for (int w = 0; w < kSbNW; w++) {
                const int r = std::min(b * kSbNW + w, nc - 1);
                lo = std::min(lo, Dc[(size_t)r * nchan + top[s]]);
            }
            for (int w = 0; w < kSbNW; w++) {
                const int r = std::min(b * kSbNW + w, nc - 1);
                const int32_t st = Dc[(size_t)r * nchan + top[s]] - lo;
                stag[(size_t)(b * kSbNW + w) * nsub + s] = st;
                maxstag = std::max(maxstag, st);
            }
        }
    for (int r = 0; r < nc; r++)
        for (int s = 0; s < nsub; s++)
            for (int c = first[s]; c < first[s + 1]; c++) {
                const int32_t v = Dc[(size_t)r * nchan + c] - stag[(size_t)r * nsub + s];
                if (v < 0) return af_set_error(AF_EINVAL, "af_plan_subband: internal stagger error");
                e[(size_t)r * nchan + c] = v;
            }
    if (int rc = af_tile_tables_build(e.data(), p->sb_cdms.data(), nc, nchan, kSbNW, kSbM, p->device, &p->sb.tile))
        return rc;
    p->sb.maxstag = maxstag;

    int maxsub = 0;
    for (int s = 0; s < nsub; s++) maxsub = std::max(maxsub, first[s + 1] - first[s]);
    p->sb.cps = (maxsub + aftile::CC - 1) / aftile::CC;
    p->sb.i16 = maxsub <= 257;  // 257 * 255 < 2^16
    const int64_t es = p->sb.i16 ? 2 : 4;
    const int64_t tv = tv_of(p->sb_n0);
    if (p->sb_L == 0) {
        int64_t L = kScratchBudget / ((int64_t)nc * nsub * es) - p->sb_rmax - 64;
        L = L / 4096 * 4096;
        p->sb_L = std::min<int64_t>(std::max<int64_t>(L, 4096), kMaxDefaultL);
    }
    p->sb.ipitch = (p->sb_L + p->sb_rmax + 7) & ~(int64_t)7;
    const size_t ibytes = ((size_t)nc * nsub * p->sb.ipitch + (size_t)tv + 64) * es;

    int rw, sc;
    size_t s2smem;
    s2_geometry(p, &rw, &sc, &s2smem);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    if (s2smem > (size_t)optin)
        return af_set_error(AF_EINVAL, "af_plan_subband: residual shifts (max %d) too large for stage 2; use a smaller n0",
                            p->sb_rmax);

    cudaError_t err;
    if ((err = cudaMalloc(&p->sb.d_stag, stag.size() * 4)) != cudaSuccess ||
        (err = cudaMemcpy(p->sb.d_stag, stag.data(), stag.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (err = cudaMalloc(&p->sb.d_first, first.size() * 4)) != cudaSuccess ||
        (err = cudaMemcpy(p->sb.d_first, first.data(), first.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (err = cudaMalloc(&p->sb.d_r, p->sb_r.size() * 4)) != cudaSuccess ||
        (err = cudaMemcpy(p->sb.d_r, p->sb_r.data(), p->sb_r.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (err = cudaMalloc(&p->sb.d_I, ibytes)) != cudaSuccess)
        return af_cuda_check(err, "af_plan_subband: device tables / scratch");
    if (p->sb.tile.fits)
        if (int rc = af_ensure_smem((const void*)aftile::k_tile_sb<kSbNW, kSbM>, af_tile_smem(kSbNW, p->sb.tile.rw)))
            return rc;
    return af_ensure_smem(p->sb.i16 ? s2_fn<uint16_t>(p->sb_n0) : s2_fn<uint32_t>(p->sb_n0), s2smem);
}

int af_launch_subband(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int64_t nout, int32_t* d_plane,
                      af_rowstats_t* d_stats, cudaStream_t s)
{
    if (d_stats)
        if (int rc = af_cuda_check(cudaMemsetAsync(d_stats, 0, (size_t)p->ndm * sizeof(af_rowstats_t), s),
                                   "subband stats reset"))
            return rc;
    constexpr int TTE = aftile::tte_of(kSbM);
    int rw, sc;
    size_t s2smem;
    s2_geometry(p, &rw, &sc, &s2smem);
    const int64_t tv = tv_of(p->sb_n0);
    const size_t s1smem = af_tile_smem(kSbNW, p->sb.tile.rw);
    if (int rc = af_ensure_smem((const void*)aftile::k_tile_sb<kSbNW, kSbM>, s1smem)) return rc;
    if (int rc = af_ensure_smem(p->sb.i16 ? s2_fn<uint16_t>(p->sb_n0) : s2_fn<uint32_t>(p->sb_n0), s2smem)) return rc;

    for (int64_t v0 = 0; v0 < nout; v0 += p->sb_L) {
        const int64_t lcur = std::min(p->sb_L, nout - v0);
        aftile::TileArgs a;
        a.X = d_in;
        a.nsamp = nsamp;
        a.total = (int64_t)p->nchan * nsamp;
        a.nchan = p->nchan;
        a.nchunks = p->sb_nsub * p->sb.cps;
        a.dsort = p->sb.tile.d_dsort;
        a.perm = p->sb.tile.d_perm;
        a.dminblk = p->sb.tile.d_dminblk;
        a.nout = 0;
        a.rw = p->sb.tile.rw;
        a.li = lcur + p->sb_rmax;
        a.tiles = (unsigned)((a.li + p->sb.maxstag + TTE - 1) / TTE);
        a.nblk = (unsigned)p->sb.tile.nblk;
        a.Y = nullptr;
        a.stats = nullptr;
        a.err = p->d_err;
        a.cps = p->sb.cps;
        a.nsub = p->sb_nsub;
        a.sbfirst = p->sb.d_first;
        a.stag = p->sb.d_stag;
        a.I = p->sb.d_I;
        a.i16 = p->sb.i16 ? 1 : 0;
        a.ipitch = p->sb.ipitch;
        a.tbase = v0;
        const unsigned long long nb1 = (unsigned long long)a.tiles * a.nblk;
        const unsigned vtiles = (unsigned)((lcur + tv - 1) / tv);
        const unsigned long long nb2 = (unsigned long long)vtiles * p->sb_ncoarse;
        if (nb1 > 0x7fffffffULL || nb2 > 0x7fffffffULL)
            return af_set_error(AF_EINVAL, "subband dedisperse: problem too large for one grid");
        aftile::k_tile_sb<kSbNW, kSbM><<<(unsigned)nb1, (kSbNW + 1) * 32, s1smem, s>>>(a);
        if (int rc = af_cuda_check(cudaGetLastError(), "subband stage 1 launch")) return rc;
        if (p->sb.i16)
            s2_launch<uint16_t>(p->sb_n0, (unsigned)nb2, s2smem, s, (const uint16_t*)p->sb.d_I, p->sb.ipitch,
                                p->sb_nsub, p->ndm, p->sb.d_r, rw, sc, v0, lcur, nout, vtiles, d_plane, d_stats,
                                p->d_err);
        else
            s2_launch<uint32_t>(p->sb_n0, (unsigned)nb2, s2smem, s, (const uint32_t*)p->sb.d_I, p->sb.ipitch,
                                p->sb_nsub, p->ndm, p->sb.d_r, rw, sc, v0, lcur, nout, vtiles, d_plane, d_stats,
                                p->d_err);
        if (int rc = af_cuda_check(cudaGetLastError(), "subband stage 2 launch")) return rc;
    }
    return AF_OK;
}
