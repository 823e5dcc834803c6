// dedisp.cu -- brute-force incoherent dedispersion (Sec. 2.3) and row sums.
//
//   Y[d][t] = sum_c X[c][t + D[d][c]],  0 <= t < nout,  exact int32.
//
// Main kernel: the tile kernel of tile.cuh (shape NW x M below), launched
// over all (DM block, time tile) pairs of the plan.
//
// Fallback kernel (k_dedisp_simple): for plans whose per-block delay spread
// does not fit the shared-memory window (very coarse DM grids); one output
// column per thread, input read through L1.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "internal.h"
#include "ptx.cuh"
#include "tile.cuh"

namespace {

// Block shape of the single-plan tile kernel (measured best on GB300).
constexpr int kDefaultNW = 11;
constexpr int kDefaultM = 8;

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

int af_ensure_smem(const void* kernel, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> set;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = set[std::make_pair(dev, kernel)];
    if (bytes <= cur) return AF_OK;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return af_cuda_check(e, "kernel shared memory attribute");
    cur = bytes;
    return AF_OK;
}

// Tile-kernel tables for one delay table and block shape: DMs sorted
// ascending (ties keep list order), padded to a multiple of nw by repeating
// the last one; the smallest delay of each block per channel; the window.
int af_tile_tables_build(const int32_t* delays, const double* dms, int ndm, int nchan, int nw, int m, int device,
                         af_tile_tables* t, std::vector<int32_t>* h_dsort, std::vector<int32_t>* h_dmin)
{
    af_tile_tables_free(t);
    std::vector<int> order(ndm);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return dms[x] < dms[y]; });
    const int nblk = (ndm + nw - 1) / nw;
    const int ndm_pad = nblk * nw;
    std::vector<int32_t> dsort((size_t)ndm_pad * nchan), perm(ndm_pad, -1), dmin((size_t)nblk * nchan);
    for (int s = 0; s < ndm_pad; s++) {
        const int src = order[s < ndm ? s : ndm - 1];
        if (s < ndm) perm[s] = src;
        std::copy(delays + (size_t)src * nchan, delays + (size_t)(src + 1) * nchan, dsort.begin() + (size_t)s * nchan);
    }
    int32_t spread = 0;
    for (int j = 0; j < nblk; j++)
        for (int c = 0; c < nchan; c++) {
            int32_t lo = INT32_MAX, hi = INT32_MIN;
            for (int w = 0; w < nw; w++) {
                const int32_t d = dsort[(size_t)(j * nw + w) * nchan + c];
                lo = std::min(lo, d);
                hi = std::max(hi, d);
            }
            dmin[(size_t)j * nchan + c] = lo;
            spread = std::max(spread, hi - lo);
        }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    t->nw = nw;
    t->m = m;
    t->ndm_pad = ndm_pad;
    t->nblk = nblk;
    t->spread = spread;
    t->rw = spread < (1 << 20) ? aftile::window_bytes(spread, m) : (1 << 20);
    t->fits = spread < (1 << 20) && af_tile_smem(nw, t->rw) <= (size_t)optin;
    t->ns1 = 0;
    for (int ns = 4; ns >= 2 && t->ns1 == 0; ns--)
        if (spread < (1 << 20) && af_tile_smem(nw, t->rw, ns) <= (size_t)optin) t->ns1 = ns;
    if (h_dsort) *h_dsort = dsort;
    if (h_dmin) *h_dmin = dmin;
    cudaError_t e;
    if ((e = cudaMalloc(&t->d_dsort, dsort.size() * 4)) != cudaSuccess ||
        (e = cudaMemcpy(t->d_dsort, dsort.data(), dsort.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&t->d_perm, perm.size() * 4)) != cudaSuccess ||
        (e = cudaMemcpy(t->d_perm, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&t->d_dminblk, dmin.size() * 4)) != cudaSuccess ||
        (e = cudaMemcpy(t->d_dminblk, dmin.data(), dmin.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess) {
        af_tile_tables_free(t);
        return af_cuda_check(e, "tile tables");
    }
    return AF_OK;
}

void af_tile_tables_free(af_tile_tables* t)
{
    cudaFree(t->d_dsort);
    cudaFree(t->d_perm);
    cudaFree(t->d_dminblk);
    t->d_dsort = nullptr;
    t->d_perm = nullptr;
    t->d_dminblk = nullptr;
    t->fits = false;
    t->ns1 = 0;
}

// The single-plan tile kernel for a ring depth (4, or 3 / 2 for wide windows).
static const void* single_kernel(int ns)
{
    return ns == 4 ? (const void*)aftile::k_tile<kDefaultNW, kDefaultM, 4>
         : ns == 3 ? (const void*)aftile::k_tile<kDefaultNW, kDefaultM, 3>
                   : (const void*)aftile::k_tile<kDefaultNW, kDefaultM, 2>;
}

int af_prepare_dedisp_tables(af_plan_t p)
{
    if (int rc = af_tile_tables_build(p->delays.data(), p->dms.data(), p->ndm, p->nchan, kDefaultNW, kDefaultM,
                                      p->device, &p->tile))
        return rc;
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_err, sizeof(int))) != cudaSuccess || (e = cudaMemset(p->d_err, 0, sizeof(int))) != cudaSuccess)
        return af_cuda_check(e, "af_plan: error flag");
    if (p->sb_nsub == 0)
        if (int rc = af_pairs_build(p)) return rc;
    if (p->tile.ns1 > 0) return af_ensure_smem(single_kernel(p->tile.ns1), af_tile_smem(kDefaultNW, p->tile.rw, p->tile.ns1));
    return AF_OK;
}

size_t af_tile_smem(int nw, int rw, int ns)
{
    return (size_t)ns * aftile::CC * rw + (size_t)ns * nw * aftile::TABW * sizeof(int) + 2 * (size_t)ns * 8;
}

int af_dedisp_tile_outputs() { return aftile::tte_of(kDefaultM); }

bool af_dedisp_uses_pairs(af_plan_t p, int64_t nout)
{
    (void)nout;  // any length: more time blocks
    return p->pairs.ok && !p->force_simple && !p->force_tile && p->sb_nsub == 0 && p->pairs.lay[0].L > 0;
}

bool af_dedisp_uses_tiles(af_plan_t p) { return p->tile.ns1 > 0 && !p->force_simple && p->sb_nsub == 0; }

int af_launch_dedisperse_tiles(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int64_t nout, int32_t* d_plane,
                               af_rowstats_t* d_stats, cudaStream_t s, unsigned tile_begin, unsigned tile_end)
{
    aftile::TileArgs a;
    a.X = d_in;
    a.nsamp = nsamp;
    a.total = (int64_t)p->nchan * nsamp;
    a.nchan = p->nchan;
    a.nchunks = (p->nchan + aftile::CC - 1) / aftile::CC;
    a.dsort = p->tile.d_dsort;
    a.perm = p->tile.d_perm;
    a.dminblk = p->tile.d_dminblk;
    a.nout = nout;
    a.rw = p->tile.rw;
    a.tiles = tile_end - tile_begin;
    a.nblk = (unsigned)p->tile.nblk;
    a.Y = d_plane;
    a.stats = d_stats;
    a.err = p->d_err;
    a.tbase = (int64_t)tile_begin * aftile::tte_of(kDefaultM);
    const unsigned long long nb = (unsigned long long)a.tiles * a.nblk;
    if (nb == 0) return AF_OK;
    if (nb > 0x7fffffffULL) return af_set_error(AF_EINVAL, "dedisperse: problem too large for one grid");
    const int ns = p->tile.ns1;
    const size_t smem = af_tile_smem(kDefaultNW, a.rw, ns);
    if (int rc = af_ensure_smem(single_kernel(ns), smem)) return rc;
    if (ns == 4)
        aftile::k_tile<kDefaultNW, kDefaultM, 4><<<(unsigned)nb, (kDefaultNW + 1) * 32, smem, s>>>(a);
    else if (ns == 3)
        aftile::k_tile<kDefaultNW, kDefaultM, 3><<<(unsigned)nb, (kDefaultNW + 1) * 32, smem, s>>>(a);
    else
        aftile::k_tile<kDefaultNW, kDefaultM, 2><<<(unsigned)nb, (kDefaultNW + 1) * 32, smem, s>>>(a);
    return af_cuda_check(cudaGetLastError(), "dedisperse launch");
}

int af_launch_dedisperse(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int64_t nout, int32_t* d_plane,
                         af_rowstats_t* d_stats, cudaStream_t s)
{
    // subband plans: the two stages, unless forced onto (or left to) the
    // brute-force kernels, which compute the same plane from the effective delays
    if (p->sb_nsub > 0 && p->sb.tile.fits && !p->force_simple && !p->force_brute)
        return af_launch_subband(p, d_in, nsamp, nout, d_plane, d_stats, s);
    if (af_dedisp_uses_pairs(p, nout)) return af_launch_pairs(p, d_in, nsamp, nout, d_plane, d_stats, s);
    if (p->tile.ns1 > 0 && !p->force_simple) {
        if (d_stats)
            if (int rc = af_cuda_check(cudaMemsetAsync(d_stats, 0, (size_t)p->ndm * sizeof(af_rowstats_t), s),
                                       "dedisperse stats reset"))
                return rc;
        const unsigned tiles = (unsigned)((nout + aftile::tte_of(kDefaultM) - 1) / aftile::tte_of(kDefaultM));
        return af_launch_dedisperse_tiles(p, d_in, nsamp, nout, d_plane, d_stats, s, 0, tiles);
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

extern "C" int af_plan_kernel(af_plan_t p, int* path, int* ring, int32_t* spread, int* group)
try {
    if (int rc = af_check_plan(p)) return rc;
    int pa = AF_PATH_SIMPLE, rg = 0, sp = p->tile.spread, gr = 1;
    if (p->sb_nsub > 0 && p->sb.tile.fits && !p->force_simple && !p->force_brute) {
        pa = AF_PATH_SUBBAND;
        rg = aftile::NSTAGE;
        sp = p->sb.tile.spread;
    } else if (af_dedisp_uses_pairs(p, 1)) {
        pa = AF_PATH_PAIRS;
        rg = af_pair_ring_depth(p->pairs.shape);
        sp = p->pairs.tt.spread;
        gr = p->pairs.G;
    } else if (p->tile.ns1 > 0 && !p->force_simple) {
        pa = AF_PATH_TILE;
        rg = p->tile.ns1;
    }
    if (path) *path = pa;
    if (ring) *ring = rg;
    if (spread) *spread = sp;
    if (group) *group = gr;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_plan_kernel");
}

int af_launch_rowstats(const int32_t* d_plane, int ndm, int64_t nout, af_rowstats_t* d_stats, cudaStream_t s)
{
    k_rowstats<<<ndm, kStatThreads, 0, s>>>(d_plane, nout, d_stats);
    return af_cuda_check(cudaGetLastError(), "rowstats launch");
}
