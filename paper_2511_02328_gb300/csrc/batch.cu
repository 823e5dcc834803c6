// batch.cu -- many beams of uneven shape dedispersed by one CUDA graph, the
// execution strategy picked by timing.
//
// af_batch_build makes one plan per beam, allocates every beam's plane, S/N
// and candidate buffers (within an HBM budget), then autotunes over the
// strategies:
//   - one persistent channel-tile launch over all (beam, DM block, time tile)
//     items, for each compiled tile shape (DM rows per block x outputs per
//     lane);
//   - the beams one after another, each on its single-plan path (group rows,
//     pairs.cu, sharing one row buffer, where the plan uses them);
//   - persistent group rows: the time axis in waves of W tiles; per wave the
//     rows of every beam's block are built (one stage-1 launch per beam, all
//     beams' rows side by side in one buffer), then ONE persistent stage-2
//     launch takes (beam, DM block, tile) items of all beams from an atomic
//     counter; tuned over W.
// Each candidate is timed on the batch itself, the fastest is kept and cached
// in a JSON file (AFGB_AUTOTUNE_CACHE) keyed by the GPU name and the beams'
// shapes.  af_batch_run replays a graph of: the dedispersion (with its
// counter and row-sum resets), then per beam the boxcar S/N and the candidate
// compaction.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"
#include "tile.cuh"

namespace {

typedef cudaError_t (*persistent_fn)(int grid, size_t smem, cudaStream_t s, const aftile::TileArgs* jobs,
                                     const long long* first, int njobs, long long total, unsigned long long* counter);
typedef cudaError_t (*attr_fn)(size_t smem);

template <int NW, int M>
cudaError_t launch_persistent(int grid, size_t smem, cudaStream_t s, const aftile::TileArgs* jobs,
                              const long long* first, int njobs, long long total, unsigned long long* counter)
{
    aftile::k_tile_persistent<NW, M><<<grid, (NW + 1) * 32, smem, s>>>(jobs, first, njobs, total, counter);
    return cudaGetLastError();
}

template <int NW, int M>
cudaError_t set_attr(size_t smem)
{
    return af_ensure_smem((const void*)aftile::k_tile_persistent<NW, M>, smem) == AF_OK ? cudaSuccess
                                                                                         : cudaErrorInvalidValue;
}

struct Shape {
    int nw, m;
    persistent_fn launch;
    attr_fn attr;
};

// Compiled block shapes the autotuner chooses from.
const Shape kShapes[] = {
    {11, 8, launch_persistent<11, 8>, set_attr<11, 8>},
    {7, 8, launch_persistent<7, 8>, set_attr<7, 8>},
    {15, 6, launch_persistent<15, 6>, set_attr<15, 6>},
};
constexpr int kNShapes = sizeof(kShapes) / sizeof(kShapes[0]);
constexpr int kPairs = kNShapes;       // strategy index of beam after beam (group rows where they apply)
constexpr int kPersist = kNShapes + 1; // strategy index of persistent group rows
constexpr size_t kPairsMax = (size_t)16 << 30;  // largest shared row buffer
constexpr size_t kPersistMax = (size_t)64 << 30;  // largest row buffer of the persistent group rows
// tiles-per-wave choices of the persistent group rows: 0 = the most the row
// buffer holds, -k = that divided by 2^k.  (The ring depth is not a choice:
// the plans' consumer tables hold shared-memory offsets of the ring stages
// they were built for, so the launch uses the plans' own depth.)
constexpr int kPersistChoices[] = {0, -1, -2};

struct Beam {
    af_plan_t plan = nullptr;
    const uint8_t* d_in = nullptr;
    int64_t nsamp = 0, nout = 0;
    af_widths_t widths;
    float thresh = 0;
    int32_t cap = 0;
    int32_t* d_plane = nullptr;
    af_rowstats_t* d_stats = nullptr;
    float* d_snr = nullptr;
    uint8_t* d_bw = nullptr;
    af_cand_t* d_cands = nullptr;
    int32_t* d_count = nullptr;
    af_tile_tables tables;
};

}  // namespace

struct af_batch_s {
    int device = 0;
    std::vector<Beam> beams;
    std::vector<int> order;              // job order (largest channel count first)
    int shape = 0;                       // index into kShapes
    float tuned_ms = 0.0f;
    bool from_cache = false;
    aftile::TileArgs* d_jobs = nullptr;
    long long* d_first = nullptr;
    unsigned long long* d_counter = nullptr;
    int* d_err = nullptr;
    long long total = 0;
    int grid = 0;
    size_t smem = 0;
    uint16_t* d_rows = nullptr;          // row buffer shared by the beams' plans (group-row strategy)
    size_t rows_bytes = 0;
    // persistent group rows
    int pp_ns = 0, pp_tiles = 0;         // ring depth, tiles per wave
    std::vector<int> pp_beam;            // per beam: 1 if on group rows
    std::vector<std::vector<int>> pp_wave_beams;  // beams with a block in each wave
    std::vector<int> pp_wave_job0;       // first job of each wave
    std::vector<long long> pp_wave_total;
    af_pair_args* d_pjobs = nullptr;
    long long* d_pfirst = nullptr;       // per wave: its jobs' item prefix (njobs + 1 entries), concatenated
    unsigned long long* d_pcounters = nullptr;
    size_t pp_smem = 0;
    uint16_t* d_prows = nullptr;
    size_t prows_bytes = 0;
    // every candidate the autotuner timed: {kind (0 tile shape, 1 beam after beam, 2 persistent rows), p1, p2, ms}
    std::vector<std::array<float, 4>> tuning;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
};

static void free_batch(af_batch_t b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (Beam& x : b->beams) {
        cudaFree(x.d_plane);
        cudaFree(x.d_stats);
        cudaFree(x.d_snr);
        cudaFree(x.d_bw);
        cudaFree(x.d_cands);
        cudaFree(x.d_count);
        af_tile_tables_free(&x.tables);
        af_plan_destroy(x.plan);
    }
    cudaFree(b->d_jobs);
    cudaFree(b->d_first);
    cudaFree(b->d_counter);
    cudaFree(b->d_err);
    cudaFree(b->d_rows);
    cudaFree(b->d_prows);
    cudaFree(b->d_pjobs);
    cudaFree(b->d_pfirst);
    cudaFree(b->d_pcounters);
    delete b;
}

// The beam-after-beam strategy: every beam on its single-plan path, group rows
// for the beams whose plans use them, all on one shared row buffer sized for
// the largest such beam's full length (at most kPairsMax; the other beams, or
// all of them past the cap, run in time blocks); the rest on the channel tile
// kernel.  AF_EINVAL: no beam can use group rows (the persistent strategies
// cover that case).
static int setup_pairs(af_batch_t b)
{
    size_t need = 0;
    std::vector<bool> use(b->beams.size(), false);
    for (size_t i = 0; i < b->beams.size(); i++) {
        Beam& x = b->beams[i];
        if (!x.plan->pairs.ok) continue;
        int64_t L = 0;  // the beam's fastest group size within the largest buffer
        if (int rc = af_pairs_pick(x.plan, x.nout, true, kPairsMax, &L)) return rc;
        if (L <= 0) continue;
        use[i] = true;
        need = std::max(need, std::min(af_pairs_bytes(x.plan, x.nout), kPairsMax));
    }
    if (need == 0) return af_set_error(AF_EINVAL, "batch: no beam gains from group rows");
    if (!b->d_rows) {
        if (cudaMalloc(&b->d_rows, need) != cudaSuccess) {
            cudaGetLastError();
            b->d_rows = nullptr;
            return af_set_error(AF_EINVAL, "batch: no room for the shared row buffer");
        }
        b->rows_bytes = need;
    }
    for (size_t i = 0; i < b->beams.size(); i++)
        if (use[i])
            if (int rc = af_pairs_attach(b->beams[i].plan, b->d_rows, b->rows_bytes, b->beams[i].nout))
                return rc == AF_ENOBUFS ? af_set_error(AF_EINVAL, "batch: shared row buffer too small") : rc;
    b->shape = kPairs;
    return AF_OK;
}

// Persistent group rows with `tiles` output tiles per wave (0: the most that
// kPersistMax of rows holds; -k: that divided by 2^k).  The launch runs a
// ring of the depth the plans' tables were built for; beams whose plans do
// not gain from group rows, or were built for another depth, run on their
// single-plan path before the waves.  AF_EINVAL: this choice does not apply
// (no such beam, or the rows of one wave do not fit).
static int setup_persist(af_batch_t b, int tiles)
{
    const int64_t tte = af_pair_tile_outputs();
    std::vector<int> use;
    int64_t max_tiles = 0;
    int ns = 0;
    for (size_t i = 0; i < b->beams.size(); i++) {
        Beam& x = b->beams[i];
        if (!x.plan->pairs.ok) continue;
        int64_t L = 0;
        if (int rc = af_pairs_pick(x.plan, x.nout, true, kPairsMax, &L)) return rc;
        if (L <= 0) continue;
        if (ns == 0) ns = af_pairs_ring(x.plan);
        if (af_pairs_ring(x.plan) != ns) continue;  // tables for another ring depth
        use.push_back((int)i);
        max_tiles = std::max(max_tiles, (x.nout + tte - 1) / tte);
    }
    if (use.empty() || ns < 2) return af_set_error(AF_EINVAL, "batch: no beam for persistent group rows");
    auto wave_bytes = [&](int64_t t, std::vector<size_t>* sizes) {
        size_t tot = 0;
        for (int i : use) {
            const Beam& x = b->beams[i];
            const size_t by = (af_pairs_bytes(x.plan, std::min(x.nout, t * tte)) + 255) & ~(size_t)255;
            if (sizes) sizes->push_back(by);
            tot += by;
        }
        return tot;
    };
    int64_t t = std::min<int64_t>(max_tiles, 8);
    if (wave_bytes(t, nullptr) > kPersistMax) return af_set_error(AF_EINVAL, "batch: one wave of rows is too large");
    if (tiles > 0) {
        t = std::max<int64_t>(t, std::min<int64_t>(tiles, max_tiles));
    } else {
        int64_t lo = t, hi = max_tiles;  // the most tiles whose rows fit
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (wave_bytes(mid, nullptr) <= kPersistMax) lo = mid;
            else hi = mid - 1;
        }
        t = std::max<int64_t>(t, lo >> (tiles < 0 ? -tiles : 0));
    }
    std::vector<size_t> sizes;
    const size_t need = wave_bytes(t, &sizes);
    if (need > b->prows_bytes) {
        if (b->d_prows) {
            if (int rc = af_cuda_check(cudaDeviceSynchronize(), "batch")) return rc;
            cudaFree(b->d_prows);
        }
        b->d_prows = nullptr;
        b->prows_bytes = 0;
        if (cudaMalloc(&b->d_prows, need) != cudaSuccess) {
            cudaGetLastError();
            b->d_prows = nullptr;
            return af_set_error(AF_EINVAL, "batch: no room for the persistent row buffer");
        }
        b->prows_bytes = need;
    }
    b->pp_beam.assign(b->beams.size(), 0);
    size_t off = 0;
    int64_t nwaves = 0;
    for (size_t k = 0; k < use.size(); k++) {
        Beam& x = b->beams[use[k]];
        if (int rc = af_pairs_attach(x.plan, b->d_prows + off / 2, sizes[k], x.nout))
            return rc == AF_ENOBUFS ? af_set_error(AF_EINVAL, "batch: persistent rows do not fit") : rc;
        off += sizes[k];
        const int64_t L = x.plan->pairs.lay[0].L;
        if (L <= 0) continue;  // the cost model keeps this beam on the channel tile kernel
        b->pp_beam[use[k]] = 1;
        nwaves = std::max(nwaves, (x.nout + L - 1) / L);
    }
    if (nwaves == 0) return af_set_error(AF_EINVAL, "batch: no beam on persistent group rows");
    std::vector<af_pair_args> jobs;
    std::vector<long long> first;
    b->pp_wave_beams.assign(nwaves, {});
    b->pp_wave_job0.assign(nwaves + 1, 0);
    b->pp_wave_total.assign(nwaves, 0);
    size_t smem = 0;
    for (int64_t w = 0; w < nwaves; w++) {
        b->pp_wave_job0[w] = (int)jobs.size();
        first.push_back(0);
        for (int k : b->order) {
            if (!b->pp_beam[k]) continue;
            Beam& x = b->beams[k];
            const int64_t L = x.plan->pairs.lay[0].L, T0 = w * L;
            if (T0 >= x.nout) continue;
            af_pair_args a;
            long long items = 0;
            if (int rc = af_pairs_block_args(x.plan, x.nout, 0, T0, x.d_plane, x.d_stats, &a, &items)) return rc;
            jobs.push_back(a);
            first.push_back(first.back() + items);
            b->pp_wave_beams[w].push_back(k);
            smem = std::max(smem, af_pairs_stage2_smem(x.plan, ns));
        }
        b->pp_wave_total[w] = first.back();
    }
    b->pp_wave_job0[nwaves] = (int)jobs.size();
    cudaFree(b->d_pjobs);
    cudaFree(b->d_pfirst);
    cudaFree(b->d_pcounters);
    b->d_pjobs = nullptr;
    b->d_pfirst = nullptr;
    b->d_pcounters = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_pjobs, jobs.size() * sizeof(af_pair_args))) != cudaSuccess ||
        (e = cudaMemcpy(b->d_pjobs, jobs.data(), jobs.size() * sizeof(af_pair_args), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMalloc(&b->d_pfirst, first.size() * sizeof(long long))) != cudaSuccess ||
        (e = cudaMemcpy(b->d_pfirst, first.data(), first.size() * sizeof(long long), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMalloc(&b->d_pcounters, (size_t)nwaves * sizeof(unsigned long long))) != cudaSuccess)
        return af_cuda_check(e, "batch: persistent job upload");
    b->pp_ns = ns;
    b->pp_tiles = (int)t;
    b->pp_smem = smem;
    b->shape = kPersist;
    return AF_OK;
}

// Builds the per-beam tile tables for shape si and uploads the job list.
static int setup_shape(af_batch_t b, int si)
{
    const Shape& sh = kShapes[si];
    int maxrw = 0;
    for (Beam& x : b->beams) {
        af_plan_t p = x.plan;
        if (int rc = af_tile_tables_build(p->delays.data(), p->dms.data(), p->ndm, p->nchan, sh.nw, sh.m, b->device,
                                          &x.tables))
            return rc;
        if (!x.tables.fits) return af_set_error(AF_EINVAL, "batch: a beam's delay spread does not fit shape %dx%d", sh.nw, sh.m);
        maxrw = std::max(maxrw, x.tables.rw);
    }
    std::vector<aftile::TileArgs> jobs;
    std::vector<long long> first(1, 0);
    for (int k : b->order) {
        const Beam& x = b->beams[k];
        aftile::TileArgs a;
        a.X = x.d_in;
        a.nsamp = x.nsamp;
        a.total = (int64_t)x.plan->nchan * x.nsamp;
        a.nchan = x.plan->nchan;
        a.nchunks = (x.plan->nchan + aftile::CC - 1) / aftile::CC;
        a.dsort = x.tables.d_dsort;
        a.perm = x.tables.d_perm;
        a.dminblk = x.tables.d_dminblk;
        a.nout = x.nout;
        a.rw = x.tables.rw;
        a.tiles = (unsigned)((x.nout + aftile::tte_of(sh.m) - 1) / aftile::tte_of(sh.m));
        a.nblk = (unsigned)x.tables.nblk;
        a.Y = x.d_plane;
        a.stats = x.d_stats;
        a.err = b->d_err;
        jobs.push_back(a);
        first.push_back(first.back() + (long long)a.tiles * a.nblk);
    }
    b->total = first.back();
    b->smem = af_tile_smem(sh.nw, maxrw);
    cudaFree(b->d_jobs);
    cudaFree(b->d_first);
    b->d_jobs = nullptr;
    b->d_first = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_jobs, jobs.size() * sizeof(aftile::TileArgs))) != cudaSuccess ||
        (e = cudaMemcpy(b->d_jobs, jobs.data(), jobs.size() * sizeof(aftile::TileArgs), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMalloc(&b->d_first, first.size() * sizeof(long long))) != cudaSuccess ||
        (e = cudaMemcpy(b->d_first, first.data(), first.size() * sizeof(long long), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = sh.attr(b->smem)) != cudaSuccess)
        return af_cuda_check(e, "batch: job upload");
    b->shape = si;
    return AF_OK;
}

static int enqueue_dedisp(af_batch_t b, cudaStream_t s)
{
    if (b->shape == kPersist) {
        const int nwaves = (int)b->pp_wave_beams.size();
        AF_CUDA(cudaMemsetAsync(b->d_pcounters, 0, (size_t)nwaves * sizeof(unsigned long long), s));
        for (int k : b->order) {
            Beam& x = b->beams[k];
            if (!b->pp_beam[k]) {  // its single-plan path
                if (int rc = af_launch_dedisperse(x.plan, x.d_in, x.nsamp, x.nout, x.d_plane, x.d_stats, s)) return rc;
            } else {
                AF_CUDA(cudaMemsetAsync(x.d_stats, 0, (size_t)x.plan->ndm * sizeof(af_rowstats_t), s));
            }
        }
        for (int w = 0; w < nwaves; w++) {
            for (int k : b->pp_wave_beams[w]) {
                Beam& x = b->beams[k];
                if (int rc = af_launch_pairs_rows(x.plan, x.d_in, x.nsamp, 0, (int64_t)w * x.plan->pairs.lay[0].L, s))
                    return rc;
            }
            const int j0 = b->pp_wave_job0[w], nj = b->pp_wave_job0[w + 1] - j0;
            if (int rc = af_launch_pairs_persistent(b->pp_ns, b->pp_smem, b->grid, b->d_pjobs + j0, b->d_pfirst + j0 + w,
                                                    nj, b->pp_wave_total[w], b->d_pcounters + w, s))
                return rc;
        }
        return AF_OK;
    }
    if (b->shape == kPairs) {
        for (int k : b->order) {
            Beam& x = b->beams[k];
            if (int rc = af_launch_dedisperse(x.plan, x.d_in, x.nsamp, x.nout, x.d_plane, x.d_stats, s)) return rc;
        }
        return AF_OK;
    }
    const Shape& sh = kShapes[b->shape];
    AF_CUDA(sh.attr(b->smem));
    AF_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), s));
    for (Beam& x : b->beams)
        AF_CUDA(cudaMemsetAsync(x.d_stats, 0, (size_t)x.plan->ndm * sizeof(af_rowstats_t), s));
    AF_CUDA(sh.launch(b->grid, b->smem, s, b->d_jobs, b->d_first, (int)b->beams.size(), b->total, b->d_counter));
    return AF_OK;
}

static int enqueue_all(af_batch_t b, cudaStream_t s)
{
    if (int rc = enqueue_dedisp(b, s)) return rc;
    for (Beam& x : b->beams) {
        if (int rc = af_launch_boxcar(x.d_plane, x.plan->ndm, x.nout, x.d_stats, x.widths, x.plan->d_rowconst,
                                      x.d_snr, x.d_bw, s))
            return rc;
        if (int rc = af_launch_candidates(x.d_snr, x.d_bw, x.plan->ndm, x.nout, x.widths, x.thresh, 0, x.d_cands,
                                          x.cap, x.d_count, s))
            return rc;
    }
    return AF_OK;
}

// ---------------------------------------------------------------- autotune cache
static std::string shape_sig(af_batch_t b)
{
    // channel count, DM list extent and sample count fix a beam's work shape
    std::string k;
    char buf[160];
    for (const Beam& x : b->beams) {
        const af_plan_s* p = x.plan;
        snprintf(buf, sizeof buf, "|%d:%d:%lld:%d:%.6g:%.6g", p->nchan, p->ndm, (long long)x.nsamp, p->dmax,
                 p->dms.front(), p->dms.back());
        k += buf;
    }
    return k;
}

static bool cache_lookup(const std::string& path, const std::string& key, int* nw, int* m)
{
    FILE* f = fopen(path.c_str(), "r");
    if (!f) return false;
    std::string txt;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, n);
    fclose(f);
    const std::string q = "\"" + key + "\"";
    size_t pos = txt.find(q);
    if (pos == std::string::npos) return false;
    size_t a = txt.find("\"nw\":", pos), c = txt.find("\"m\":", pos);
    if (a == std::string::npos || c == std::string::npos) return false;
    *nw = atoi(txt.c_str() + a + 5);
    *m = atoi(txt.c_str() + c + 4);
    return true;
}

static void cache_store(const std::string& path, const std::string& key, int nw, int m, float ms)
{
    std::string txt;
    if (FILE* f = fopen(path.c_str(), "r")) {
        char buf[4096];
        size_t n;
        while ((n = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, n);
        fclose(f);
    }
    // keep the object's existing entries, append the new one
    size_t end = txt.rfind('}');
    char entry[256];
    snprintf(entry, sizeof entry, "{\"nw\": %d, \"m\": %d, \"ms\": %.4f}", nw, m, ms);
    std::string item = "\"" + key + "\": " + entry;
    if (end == std::string::npos || txt.find('{') == std::string::npos) {
        txt = "{\n  " + item + "\n}\n";
    } else {
        bool empty = txt.find('"') == std::string::npos;
        txt = txt.substr(0, end) + (empty ? "  " : ",\n  ") + item + "\n}\n";
    }
    std::string tmp = path + ".tmp";
    if (FILE* f = fopen(tmp.c_str(), "w")) {
        fwrite(txt.data(), 1, txt.size(), f);
        fclose(f);
        rename(tmp.c_str(), path.c_str());
    }
}

// One candidate strategy: kind 0 = persistent channel tiles (shape p1),
// 1 = beam after beam, 2 = persistent group rows (ring p1, tiles per wave p2).
struct Cand {
    int kind, p1, p2;
};

static int setup_cand(af_batch_t b, const Cand& c)
{
    return c.kind == 0 ? setup_shape(b, c.p1) : c.kind == 1 ? setup_pairs(b) : setup_persist(b, c.p2);
}

// Back to no group-row layout on any plan, and free the row buffers the
// candidate `keep` (kind) does not use.
static int release_rows(af_batch_t b, int keep)
{
    if (int r = af_cuda_check(cudaDeviceSynchronize(), "batch")) return r;
    for (Beam& x : b->beams) x.plan->pairs.lay[0].L = x.plan->pairs.lay[1].L = 0;
    if (keep != 1 && b->d_rows) {
        cudaFree(b->d_rows);
        b->d_rows = nullptr;
        b->rows_bytes = 0;
    }
    if (keep != 2 && b->d_prows) {
        cudaFree(b->d_prows);
        b->d_prows = nullptr;
        b->prows_bytes = 0;
    }
    return AF_OK;
}

static int autotune(af_batch_t b)
{
    const char* path = getenv("AFGB_AUTOTUNE_CACHE");
    const std::string key = [&] {
        cudaDeviceProp prop;
        cudaGetDeviceProperties(&prop, b->device);
        return std::string(prop.name) + shape_sig(b);
    }();
    if (path) {
        int nw = 0, m = 0;
        if (cache_lookup(path, key, &nw, &m)) {
            // m > 0: tile shape (nw, m); m == 0: beam after beam; m < 0: persistent rows (ring nw, -m tiles)
            Cand c{-1, 0, 0};
            if (m == 0) c = Cand{1, 0, 0};
            else if (m < 0) c = Cand{2, nw, -m};  // the tiles per wave it resolved to
            else
                for (int si = 0; si < kNShapes; si++)
                    if (kShapes[si].nw == nw && kShapes[si].m == m) c = Cand{0, si, 0};
            if (c.kind >= 0) {
                if (int rc = setup_cand(b, c)) return rc;
                b->from_cache = true;
                return AF_OK;
            }
        }
    }
    // AFGB_BATCH_STRATEGY=tile|pairs|persistent restricts the candidates
    const char* only = getenv("AFGB_BATCH_STRATEGY");
    std::vector<Cand> cands;
    if (!only || !strcmp(only, "tile"))
        for (int si = 0; si < kNShapes; si++) cands.push_back(Cand{0, si, 0});
    if (!only || !strcmp(only, "pairs")) cands.push_back(Cand{1, 0, 0});
    if (!only || !strcmp(only, "persistent"))
        for (int tc : kPersistChoices) cands.push_back(Cand{2, 0, tc});
    cudaStream_t s;
    AF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = -1;
    Cand best_c{0, 0, 0};
    float best_ms = 0.0f;
    int rc = AF_OK;
    b->tuning.clear();
    for (size_t ci = 0; ci < cands.size() && rc == AF_OK; ci++) {
        Cand c = cands[ci];
        int r = setup_cand(b, c);
        if (r == AF_EINVAL) continue;  // this candidate does not apply to these beams: skip it
        if (r) {
            rc = r;
            break;
        }
        if (c.kind == 2) c.p1 = b->pp_ns, c.p2 = b->pp_tiles;  // what it resolved to
        float ms = 0.0f;
        for (int rep = 0; rep < 3 && rc == AF_OK; rep++) {
            cudaEventRecord(e0, s);
            rc = enqueue_dedisp(b, s);
            cudaEventRecord(e1, s);
            cudaError_t ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) rc = af_cuda_check(ce, "autotune");
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms += t / 2.0f;  // first run warms up
        }
        if (rc != AF_OK) break;
        b->tuning.push_back({(float)c.kind, (float)(c.kind == 0 ? kShapes[c.p1].nw : c.p1),
                             (float)(c.kind == 0 ? kShapes[c.p1].m : c.p2), ms});
        if (best < 0 || ms < best_ms) {
            best = (int)ci;
            best_c = c;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (rc) return rc;
    if (best < 0) return af_set_error(AF_EINVAL, "batch: no strategy fits these beams");
    if (int r = release_rows(b, best_c.kind)) return r;
    if (int r = setup_cand(b, best_c)) return r;
    b->tuned_ms = best_ms;
    if (path) {
        const int nw = best_c.kind == 0 ? kShapes[best_c.p1].nw : best_c.kind == 1 ? 15 : best_c.p1;
        const int m = best_c.kind == 0 ? kShapes[best_c.p1].m : best_c.kind == 1 ? 0 : -best_c.p2;
        cache_store(path, key, nw, m, best_ms);
    }
    return AF_OK;
}

extern "C" int af_batch_build(af_batch_t* out, const af_beam_desc_t* beams, int nbeams, size_t hbm_budget)
try {
    if (!out || !beams || nbeams < 1 || nbeams > 4096) return af_set_error(AF_EINVAL, "af_batch_build: bad arguments");
    *out = nullptr;
    af_batch_s* b = new (std::nothrow) af_batch_s();
    if (!b) return af_set_error(AF_ENOMEM, "af_batch_build: host allocation failed");
    cudaGetDevice(&b->device);
    b->beams.resize(nbeams);
    size_t bytes = 0;
    int rc = AF_OK;
    for (int i = 0; i < nbeams && rc == AF_OK; i++) {
        const af_beam_desc_t& d = beams[i];
        Beam& x = b->beams[i];
        if (!d.d_in || ((uintptr_t)d.d_in & 15)) {
            rc = af_set_error(AF_EINVAL, "af_batch_build: beam %d input NULL or not 16-byte aligned", i);
            break;
        }
        if ((rc = af_plan(&x.plan, d.nchan, d.f_lo, d.f_hi, d.tsamp, d.dm_list, d.ndm))) break;
        x.d_in = d.d_in;
        x.nsamp = d.nsamp;
        if ((rc = af_plan_nout(x.plan, d.nsamp, &x.nout))) break;
        if ((rc = af_check_widths(x.plan, d.widths, d.nw, x.nout, &x.widths))) break;
        if (d.cap < 1 || !isfinite(d.thresh)) {
            rc = af_set_error(AF_EINVAL, "af_batch_build: beam %d capacity or threshold", i);
            break;
        }
        x.thresh = d.thresh;
        x.cap = d.cap;
        const size_t npl = (size_t)d.ndm * (size_t)x.nout;
        bytes += npl * 9 + (size_t)d.ndm * sizeof(af_rowstats_t) + (size_t)d.cap * sizeof(af_cand_t) +
                 (size_t)d.ndm * d.nchan * 8;
        if (hbm_budget && bytes > hbm_budget) {
            rc = af_set_error(AF_ENOBUFS, "af_batch_build: %zu bytes needed by %d beams exceed the budget of %zu",
                              bytes, i + 1, hbm_budget);
            break;
        }
        cudaError_t e;
        if ((e = cudaMalloc(&x.d_plane, npl * 4)) != cudaSuccess || (e = cudaMalloc(&x.d_snr, npl * 4)) != cudaSuccess ||
            (e = cudaMalloc(&x.d_bw, npl)) != cudaSuccess ||
            (e = cudaMalloc(&x.d_stats, (size_t)d.ndm * sizeof(af_rowstats_t))) != cudaSuccess ||
            (e = cudaMalloc(&x.d_cands, (size_t)d.cap * sizeof(af_cand_t))) != cudaSuccess ||
            (e = cudaMalloc(&x.d_count, 16)) != cudaSuccess)
            rc = af_cuda_check(e, "af_batch_build: beam buffers");
    }
    if (rc == AF_OK) {
        cudaError_t e;
        if ((e = cudaMalloc(&b->d_counter, sizeof(unsigned long long))) != cudaSuccess ||
            (e = cudaMalloc(&b->d_err, sizeof(int))) != cudaSuccess || (e = cudaMemset(b->d_err, 0, sizeof(int))) != cudaSuccess)
            rc = af_cuda_check(e, "af_batch_build: counters");
    }
    if (rc == AF_OK) {
        b->order.resize(nbeams);
        std::iota(b->order.begin(), b->order.end(), 0);
        std::stable_sort(b->order.begin(), b->order.end(),
                         [&](int p, int q) { return b->beams[p].plan->nchan > b->beams[q].plan->nchan; });
        int nsm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
        b->grid = nsm;  // one resident block per SM (shared memory and registers allow one)
        rc = autotune(b);
    }
    if (rc != AF_OK) {
        free_batch(b);
        return rc;
    }
    *out = b;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_batch_build");
}

extern "C" int af_batch_run(af_batch_t b, void* stream)
try {
    if (!b) return af_set_error(AF_EINVAL, "af_batch_run: NULL batch");
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->exec) {
        // capture once on a private stream, then replay on the caller's
        cudaStream_t cs;
        AF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        int rc = e == cudaSuccess ? enqueue_all(b, cs) : af_cuda_check(e, "af_batch_run: begin capture");
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e2 != cudaSuccess) return af_cuda_check(e2, "af_batch_run: end capture");
        b->graph = g;
        AF_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
    }
    AF_CUDA(cudaGraphLaunch(b->exec, s));
    return AF_OK;
} catch (...) {
    return af_host_exception("af_batch_run");
}

extern "C" int af_batch_candidates(af_batch_t b, int beam, af_cand_t* h_out, int32_t cap, int32_t* h_count)
try {
    if (!b || beam < 0 || beam >= (int)b->beams.size() || !h_count || (cap > 0 && !h_out))
        return af_set_error(AF_EINVAL, "af_batch_candidates: bad arguments");
    Beam& x = b->beams[beam];
    int32_t total = 0;
    AF_CUDA(cudaMemcpy(&total, x.d_count, sizeof(int32_t), cudaMemcpyDeviceToHost));
    int flag = 0;
    AF_CUDA(cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        cudaMemset(b->d_err, 0, sizeof(int));
        return af_set_error(AF_ETIMEOUT, "af_batch: a kernel's bounded wait for an asynchronous copy ran out");
    }
    if (b->shape == kPairs || b->shape == kPersist)
        if (int rc = af_plan_check(x.plan)) return rc;  // the pair kernels flag on the beam's plan
    int32_t n = std::min(std::min(total, cap), x.cap);
    if (n > 0) {
        AF_CUDA(cudaMemcpy(h_out, x.d_cands, (size_t)n * sizeof(af_cand_t), cudaMemcpyDeviceToHost));
        std::sort(h_out, h_out + n, [](const af_cand_t& p, const af_cand_t& q) {
            return p.dm_idx != q.dm_idx ? p.dm_idx < q.dm_idx : p.t < q.t;
        });
    }
    *h_count = total;
    if (total > std::min(cap, x.cap)) return af_set_error(AF_EOVERFLOW, "af_batch_candidates: %d found", total);
    return AF_OK;
} catch (...) {
    return af_host_exception("af_batch_candidates");
}

extern "C" int af_batch_buffers(af_batch_t b, int beam, int32_t** d_plane, float** d_snr, uint8_t** d_bw,
                                int64_t* nout)
try {
    if (!b || beam < 0 || beam >= (int)b->beams.size()) return af_set_error(AF_EINVAL, "af_batch_buffers: bad beam");
    Beam& x = b->beams[beam];
    if (d_plane) *d_plane = x.d_plane;
    if (d_snr) *d_snr = x.d_snr;
    if (d_bw) *d_bw = x.d_bw;
    if (nout) *nout = x.nout;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_batch_buffers");
}

extern "C" int af_batch_shape(af_batch_t b, int* nw, int* m, float* tuned_ms, int* from_cache)
try {
    if (!b) return af_set_error(AF_EINVAL, "af_batch_shape: NULL batch");
    // persistent channel tiles: the shape; beam after beam: (15, 0); persistent
    // group rows: (ring depth, -tiles per wave)
    if (nw) *nw = b->shape == kPairs ? 15 : b->shape == kPersist ? b->pp_ns : kShapes[b->shape].nw;
    if (m) *m = b->shape == kPairs ? 0 : b->shape == kPersist ? -b->pp_tiles : kShapes[b->shape].m;
    if (tuned_ms) *tuned_ms = b->tuned_ms;
    if (from_cache) *from_cache = b->from_cache ? 1 : 0;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_batch_shape");
}

extern "C" int af_batch_tuning(af_batch_t b, int i, int* kind, int* p1, int* p2, float* ms)
try {
    if (!b || i < 0 || i >= (int)b->tuning.size() || !kind || !p1 || !p2 || !ms)
        return af_set_error(AF_EINVAL, "af_batch_tuning: bad arguments or no candidate %d", i);
    const auto& t = b->tuning[i];
    *kind = (int)t[0];
    *p1 = (int)t[1];
    *p2 = (int)t[2];
    *ms = t[3];
    return AF_OK;
} catch (...) {
    return af_host_exception("af_batch_tuning");
}

extern "C" int af_batch_destroy(af_batch_t b)
try {
    free_batch(b);
    return AF_OK;
} catch (...) {
    return af_host_exception("af_batch_destroy");
}
