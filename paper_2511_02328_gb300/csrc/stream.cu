// stream.cu -- streaming search engine with continuous batching.
//
// Each beam is a continuous 8-bit filterbank stream.  It is searched in
// windows of `window` samples that start every hop = window - Dmax samples,
// so consecutive windows overlap by the largest delay Dmax and their output
// spans (nout = hop samples each) tile the stream exactly -- the time blocking
// with a halo of the paper's Eq. (L1), Sec. 2.3, applied across chunks.  The
// last Dmax samples of every beam stay on the device between windows.
//
// Requests (one window of one beam) are admitted into slots; the number of
// slots is set by an HBM budget.  A dispatcher thread takes every window whose
// input is on the device and runs them together -- their dedispersion (on
// group rows, pairs.cu, window after window on the plan's row buffer where the
// plan uses them and the budget holds the buffer; else one persistent
// channel-tile launch over all their (DM block, time tile) items), then each
// window's boxcar S/N and candidate compaction, then the candidates' copy to
// pinned host memory.  Windows that arrive while others run are admitted as
// slots free up and join the next launch, so copies and computation of
// different requests overlap on the device.  A host callback stamps each
// window's completion; latency = completion - arrival (push call).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"
#include "tile.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kNW = 11, kM = 8;   // tile shape of the plan's tables (the single-plan default)

enum SlotState { FREE, FILLING, READY, RUNNING, DONE, HELD };

struct Slot {
    SlotState state = FREE;
    int beam = -1;
    int64_t seq = 0, sample0 = 0;
    Clock::time_point t_push, t_done;
    cudaStream_t stream = nullptr;
    cudaEvent_t input_ready = nullptr;
    uint8_t* d_in = nullptr;
    int32_t* d_plane = nullptr;
    af_rowstats_t* d_stats = nullptr;
    float* d_snr = nullptr;
    uint8_t* d_bw = nullptr;
    af_cand_t* d_cands = nullptr;
    int32_t* d_count = nullptr;
    af_cand_t* h_cands = nullptr;  // pinned
    int32_t* h_count = nullptr;    // pinned
};

struct BeamState {
    uint8_t* d_overlap = nullptr;  // [nchan][dmax]: the last dmax samples of the stream
    bool started = false;
    int64_t next_seq = 0;
    int64_t next_sample = 0;       // stream index of the first sample of the next window
    cudaEvent_t overlap_ready = nullptr;
};

}  // namespace

struct af_stream_s;

struct DoneArg {
    af_stream_s* s;
    int slot;
};

struct af_stream_s {
    af_plan_t plan = nullptr;
    int nbeams = 0, nchan = 0, ndm = 0;
    int64_t window = 0, hop = 0, dmax = 0;
    af_widths_t widths;
    float thresh = 0;
    int32_t cap = 0;
    int timeout_ms = 0;
    std::vector<Slot> slots;
    std::vector<BeamState> beams;
    std::vector<DoneArg> done_args;

    // dispatcher
    std::mutex mu;
    std::condition_variable cv_ready, cv_free, cv_done;
    std::deque<int> ready, done;
    std::thread thr;
    bool stop = false;
    int error = AF_OK;
    std::string error_msg;               // the cause, recorded by the thread that set `error`
    cudaStream_t dstream = nullptr;
    // job buffers for the persistent launches (ring)
    static constexpr int kRing = 8;
    aftile::TileArgs* h_jobs[kRing] = {};
    aftile::TileArgs* d_jobs[kRing] = {};
    long long* h_first[kRing] = {};
    long long* d_first[kRing] = {};
    cudaEvent_t ring_free[kRing] = {};
    int ring_pos = 0;
    unsigned long long* d_counter = nullptr;
    int* d_err = nullptr;
    int grid = 0;
    size_t smem = 0;
    bool pairs = false;                  // windows dedispersed on group rows
    int max_batch = 0;
    // inline classification of held windows
    cudaStream_t cstream = nullptr;
    af_cand_t* d_ccands = nullptr;
    float* d_cprob = nullptr;

    // statistics
    std::vector<double> lat_ms;
    int64_t windows_done = 0;
    int max_inflight = 0, inflight = 0;
    Clock::time_point t_first;
    bool have_first = false;
    Clock::time_point t_last;
    int64_t launches = 0;
};

static void CUDART_CB on_done(void* p)
{
    DoneArg* a = (DoneArg*)p;
    af_stream_s* s = a->s;
    std::lock_guard<std::mutex> lk(s->mu);
    Slot& sl = s->slots[a->slot];
    sl.t_done = Clock::now();
    sl.state = DONE;
    try {  // runs on a CUDA callback thread: nothing may throw out of it
        s->done.push_back(a->slot);
    } catch (...) {
        s->error = AF_ENOMEM;
        s->error_msg.clear();
        try {
            s->error_msg = "host allocation failed in the completion callback";
        } catch (...) {
        }
    }
    s->cv_done.notify_all();
}

static int dispatch(af_stream_s* s, const std::vector<int>& batch)
{
    af_plan_t p = s->plan;
    const int r = s->ring_pos;
    s->ring_pos = (s->ring_pos + 1) % af_stream_s::kRing;
    AF_CUDA(cudaEventSynchronize(s->ring_free[r]));  // the launch that used this buffer has finished
    aftile::TileArgs* jobs = s->h_jobs[r];
    long long* first = s->h_first[r];
    first[0] = 0;
    const unsigned tiles = (unsigned)((s->hop + aftile::tte_of(kM) - 1) / aftile::tte_of(kM));
    for (size_t i = 0; i < batch.size(); i++) {
        Slot& sl = s->slots[batch[i]];
        aftile::TileArgs a;
        a.X = sl.d_in;
        a.nsamp = s->window;
        a.total = (int64_t)s->nchan * s->window;
        a.nchan = s->nchan;
        a.nchunks = (s->nchan + aftile::CC - 1) / aftile::CC;
        a.dsort = p->tile.d_dsort;
        a.perm = p->tile.d_perm;
        a.dminblk = p->tile.d_dminblk;
        a.nout = s->hop;
        a.rw = p->tile.rw;
        a.tiles = tiles;
        a.nblk = (unsigned)p->tile.nblk;
        a.Y = sl.d_plane;
        a.stats = sl.d_stats;
        a.err = s->d_err;
        jobs[i] = a;
        first[i + 1] = first[i] + (long long)tiles * a.nblk;
    }
    cudaStream_t d = s->dstream;
    if (s->pairs) {
        // window after window on the plan's row buffer (one stream: no overlap between them)
        for (int k : batch) {
            Slot& sl = s->slots[k];
            AF_CUDA(cudaStreamWaitEvent(d, sl.input_ready, 0));
            if (int rc = af_launch_pairs(p, sl.d_in, s->window, s->hop, sl.d_plane, sl.d_stats, d)) return rc;
        }
    } else {
    AF_CUDA(cudaMemcpyAsync(s->d_jobs[r], jobs, batch.size() * sizeof(aftile::TileArgs), cudaMemcpyHostToDevice, d));
    AF_CUDA(cudaMemcpyAsync(s->d_first[r], first, (batch.size() + 1) * sizeof(long long), cudaMemcpyHostToDevice, d));
    for (int k : batch) AF_CUDA(cudaStreamWaitEvent(d, s->slots[k].input_ready, 0));
    AF_CUDA(cudaMemsetAsync(s->d_counter, 0, sizeof(unsigned long long), d));
    for (int k : batch) AF_CUDA(cudaMemsetAsync(s->slots[k].d_stats, 0, (size_t)s->ndm * sizeof(af_rowstats_t), d));
    if (int rc = af_ensure_smem((const void*)aftile::k_tile_persistent<kNW, kM>, s->smem)) return rc;
    aftile::k_tile_persistent<kNW, kM><<<s->grid, (kNW + 1) * 32, s->smem, d>>>(
        s->d_jobs[r], s->d_first[r], (int)batch.size(), first[batch.size()], s->d_counter);
    AF_CUDA(cudaGetLastError());
    }
    AF_CUDA(cudaEventRecord(s->ring_free[r], d));
    for (int k : batch) {
        Slot& sl = s->slots[k];
        if (int rc = af_launch_boxcar(sl.d_plane, s->ndm, s->hop, sl.d_stats, s->widths, p->d_rowconst, sl.d_snr,
                                      sl.d_bw, d))
            return rc;
        if (int rc = af_launch_candidates(sl.d_snr, sl.d_bw, s->ndm, s->hop, s->widths, s->thresh, sl.sample0,
                                          sl.d_cands, s->cap, sl.d_count, d))
            return rc;
        AF_CUDA(cudaMemcpyAsync(sl.h_count, sl.d_count, sizeof(int32_t), cudaMemcpyDeviceToHost, d));
        AF_CUDA(cudaMemcpyAsync(sl.h_cands, sl.d_cands, (size_t)s->cap * sizeof(af_cand_t), cudaMemcpyDeviceToHost, d));
        AF_CUDA(cudaLaunchHostFunc(d, on_done, &s->done_args[k]));
    }
    s->launches++;
    return AF_OK;
}

static void dispatcher(af_stream_s* s)
{
    cudaSetDevice(s->plan->device);
    for (;;) {
        int rc = AF_OK;
        try {  // a host exception becomes the engine's error status, as a failed dispatch does
            std::vector<int> batch;
            {
                std::unique_lock<std::mutex> lk(s->mu);
                s->cv_ready.wait(lk, [&] { return s->stop || !s->ready.empty(); });
                if (s->ready.empty() && s->stop) return;
                while (!s->ready.empty() && (int)batch.size() < s->max_batch) {
                    batch.push_back(s->ready.front());
                    s->ready.pop_front();
                }
                for (int k : batch) s->slots[k].state = RUNNING;
            }
            rc = dispatch(s, batch);
        } catch (...) {
            rc = af_host_exception("af_stream dispatcher");
        }
        if (rc != AF_OK) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->error = rc;
            try {  // this thread's af_last_error() holds the cause; keep it for push / poll
                s->error_msg = af_last_error();
            } catch (...) {
            }
            s->cv_done.notify_all();
            s->cv_free.notify_all();
        }
    }
}

static void free_stream(af_stream_s* s)
{
    if (!s) return;
    if (s->thr.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_ready.notify_all();
        s->thr.join();
    }
    if (s->dstream) cudaStreamSynchronize(s->dstream);
    for (Slot& sl : s->slots) {
        if (sl.stream) {
            cudaStreamSynchronize(sl.stream);
            cudaStreamDestroy(sl.stream);
        }
        if (sl.input_ready) cudaEventDestroy(sl.input_ready);
        cudaFree(sl.d_in);
        cudaFree(sl.d_plane);
        cudaFree(sl.d_stats);
        cudaFree(sl.d_snr);
        cudaFree(sl.d_bw);
        cudaFree(sl.d_cands);
        cudaFree(sl.d_count);
        cudaFreeHost(sl.h_cands);
        cudaFreeHost(sl.h_count);
    }
    for (BeamState& b : s->beams) {
        cudaFree(b.d_overlap);
        if (b.overlap_ready) cudaEventDestroy(b.overlap_ready);
    }
    for (int r = 0; r < af_stream_s::kRing; r++) {
        cudaFreeHost(s->h_jobs[r]);
        cudaFreeHost(s->h_first[r]);
        cudaFree(s->d_jobs[r]);
        cudaFree(s->d_first[r]);
        if (s->ring_free[r]) cudaEventDestroy(s->ring_free[r]);
    }
    cudaFree(s->d_counter);
    cudaFree(s->d_err);
    cudaFree(s->d_ccands);
    cudaFree(s->d_cprob);
    if (s->cstream) cudaStreamDestroy(s->cstream);
    if (s->dstream) cudaStreamDestroy(s->dstream);
    af_plan_destroy(s->plan);
    delete s;
}

extern "C" int af_stream_open(af_stream_t* out, const af_stream_cfg_t* cfg)
try {
    if (!out || !cfg) return af_set_error(AF_EINVAL, "af_stream_open: NULL argument");
    *out = nullptr;
    if (cfg->nbeams < 1 || cfg->nbeams > 4096) return af_set_error(AF_EINVAL, "af_stream_open: nbeams");
    if (cfg->cap < 1 || !isfinite(cfg->thresh)) return af_set_error(AF_EINVAL, "af_stream_open: cap or thresh");
    af_stream_s* s = new (std::nothrow) af_stream_s();
    if (!s) return af_set_error(AF_ENOMEM, "af_stream_open: host allocation");
    int rc = af_plan(&s->plan, cfg->nchan, cfg->f_lo, cfg->f_hi, cfg->tsamp, cfg->dm_list, cfg->ndm);
    if (rc) {
        delete s;
        return rc;
    }
    af_plan_t p = s->plan;
    s->nbeams = cfg->nbeams;
    s->nchan = cfg->nchan;
    s->ndm = cfg->ndm;
    s->window = cfg->window;
    s->dmax = p->dmax;
    s->hop = cfg->window - p->dmax;
    s->thresh = cfg->thresh;
    s->cap = cfg->cap;
    s->timeout_ms = cfg->timeout_ms;
    if (s->hop < 1 || s->hop > INT32_MAX) rc = af_set_error(AF_EINVAL, "af_stream_open: window must exceed Dmax %d", p->dmax);
    if (!rc) rc = af_check_widths(p, cfg->widths, cfg->nw, s->hop, &s->widths);
    if (rc) {
        free_stream(s);
        return rc;
    }
    const size_t slot_bytes = (size_t)s->nchan * s->window + (size_t)s->ndm * s->hop * 9 +
                              (size_t)s->ndm * sizeof(af_rowstats_t) + (size_t)s->cap * sizeof(af_cand_t) + 64;
    const size_t beam_bytes = (size_t)s->nchan * (size_t)std::max<int64_t>(s->dmax, 1);
    size_t budget = cfg->hbm_budget;
    // the group-row buffer, where the plan uses group rows: the fastest group
    // size whose buffer the budget holds next to the beam state and one slot
    size_t rows = 0;
    if (p->pairs.ok && !p->force_tile && !p->force_simple) {
        const size_t fixed = beam_bytes * s->nbeams + slot_bytes;
        if (!budget || budget > fixed) {
            if ((rc = af_pairs_reserve(p, s->hop, false, true, budget ? budget - fixed : SIZE_MAX))) {
                free_stream(s);
                return rc;
            }
            s->pairs = af_dedisp_uses_pairs(p, s->hop);
            if (s->pairs) rows = p->pairs.ps_bytes;
        }
    }
    if (!s->pairs && !p->tile.fits) {
        free_stream(s);
        return af_set_error(AF_EINVAL, "af_stream_open: DM grid too coarse for the tile kernel");
    }
    int nslots = cfg->max_slots > 0 ? cfg->max_slots : 4;
    if (budget) {
        if (budget < beam_bytes * s->nbeams + slot_bytes + rows) {
            free_stream(s);
            return af_set_error(AF_ENOBUFS, "af_stream_open: budget %zu below one slot (%zu) + beam state (%zu)",
                                budget, slot_bytes, beam_bytes * s->nbeams);
        }
        nslots = std::min<int64_t>(nslots, (budget - beam_bytes * s->nbeams - rows) / slot_bytes);
    }
    s->max_batch = nslots;
    s->slots.resize(nslots);
    s->done_args.resize(nslots);
    s->beams.resize(s->nbeams);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < nslots && e == cudaSuccess; i++) {
        Slot& sl = s->slots[i];
        s->done_args[i] = DoneArg{s, i};
        if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&sl.input_ready, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaMalloc(&sl.d_in, (size_t)s->nchan * s->window)) != cudaSuccess ||
            (e = cudaMalloc(&sl.d_plane, (size_t)s->ndm * s->hop * 4)) != cudaSuccess ||
            (e = cudaMalloc(&sl.d_snr, (size_t)s->ndm * s->hop * 4)) != cudaSuccess ||
            (e = cudaMalloc(&sl.d_bw, (size_t)s->ndm * s->hop)) != cudaSuccess ||
            (e = cudaMalloc(&sl.d_stats, (size_t)s->ndm * sizeof(af_rowstats_t))) != cudaSuccess ||
            (e = cudaMalloc(&sl.d_cands, (size_t)s->cap * sizeof(af_cand_t))) != cudaSuccess ||
            (e = cudaMalloc(&sl.d_count, 16)) != cudaSuccess ||
            (e = cudaMallocHost(&sl.h_cands, (size_t)s->cap * sizeof(af_cand_t))) != cudaSuccess ||
            (e = cudaMallocHost(&sl.h_count, 16)) != cudaSuccess)
            break;
    }
    for (int b = 0; b < s->nbeams && e == cudaSuccess; b++) {
        if ((e = cudaMalloc(&s->beams[b].d_overlap, beam_bytes)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s->beams[b].overlap_ready, cudaEventDisableTiming)) != cudaSuccess)
            break;
    }
    for (int r = 0; r < af_stream_s::kRing && e == cudaSuccess; r++) {
        if ((e = cudaMallocHost(&s->h_jobs[r], (size_t)nslots * sizeof(aftile::TileArgs))) != cudaSuccess ||
            (e = cudaMallocHost(&s->h_first[r], (size_t)(nslots + 1) * sizeof(long long))) != cudaSuccess ||
            (e = cudaMalloc(&s->d_jobs[r], (size_t)nslots * sizeof(aftile::TileArgs))) != cudaSuccess ||
            (e = cudaMalloc(&s->d_first[r], (size_t)(nslots + 1) * sizeof(long long))) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s->ring_free[r], cudaEventDisableTiming)) != cudaSuccess)
            break;
    }
    if (e == cudaSuccess && (e = cudaMalloc(&s->d_counter, 16)) == cudaSuccess &&
        (e = cudaMalloc(&s->d_err, 16)) == cudaSuccess && (e = cudaMemset(s->d_err, 0, 16)) == cudaSuccess &&
        (e = cudaMalloc(&s->d_ccands, (size_t)s->cap * sizeof(af_cand_t))) == cudaSuccess &&
        (e = cudaMalloc(&s->d_cprob, (size_t)s->cap * sizeof(float))) == cudaSuccess &&
        (e = cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking)) == cudaSuccess)
        e = cudaStreamCreateWithFlags(&s->dstream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !s->pairs) {
        s->smem = af_tile_smem(kNW, p->tile.rw);
        if (af_ensure_smem((const void*)aftile::k_tile_persistent<kNW, kM>, s->smem) != AF_OK)
            e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) {
        rc = af_cuda_check(e, "af_stream_open: allocation");
        free_stream(s);
        return rc;
    }
    cudaDeviceGetAttribute(&s->grid, cudaDevAttrMultiProcessorCount, p->device);
    s->thr = std::thread(dispatcher, s);
    *out = s;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_stream_open");
}

extern "C" int af_stream_push(af_stream_t s, int beam, const uint8_t* h_data, int64_t nsamp, int64_t pitch,
                               int64_t seq)
try {
    if (!s || !h_data || beam < 0 || beam >= s->nbeams) return af_set_error(AF_EINVAL, "af_stream_push: bad arguments");
    if (pitch == 0) pitch = nsamp;
    if (pitch < nsamp) return af_set_error(AF_EINVAL, "af_stream_push: pitch %lld < nsamp %lld", (long long)pitch, (long long)nsamp);
    const Clock::time_point t_arrive = Clock::now();
    int k = -1;
    int64_t sample0 = 0;
    bool first = false;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->error) return af_set_error(s->error, "af_stream_push: the engine failed earlier: %s", s->error_msg.c_str());
        BeamState& b = s->beams[beam];
        if (seq != b.next_seq)
            return af_set_error(AF_EINVAL, "af_stream_push: beam %d expects chunk %lld, got %lld (dropped or repeated)",
                                beam, (long long)b.next_seq, (long long)seq);
        first = !b.started;
        const int64_t want = first ? s->window : s->hop;
        if (nsamp != want)
            return af_set_error(AF_EINVAL, "af_stream_push: beam %d chunk %lld has %lld samples, expected %lld", beam,
                                (long long)seq, (long long)nsamp, (long long)want);
        auto has_free = [&] {
            for (size_t i = 0; i < s->slots.size(); i++)
                if (s->slots[i].state == FREE) return true;
            return false;
        };
        if (!has_free()) {
            if (s->timeout_ms <= 0) return af_set_error(AF_EAGAIN, "af_stream_push: no free slot");
            if (!s->cv_free.wait_for(lk, std::chrono::milliseconds(s->timeout_ms),
                                     [&] { return has_free() || s->error; }))
                return af_set_error(AF_ETIMEOUT, "af_stream_push: no slot freed within %d ms", s->timeout_ms);
            if (s->error) return af_set_error(s->error, "af_stream_push: the engine failed: %s", s->error_msg.c_str());
        }
        for (size_t i = 0; i < s->slots.size(); i++)
            if (s->slots[i].state == FREE) {
                k = (int)i;
                break;
            }
        Slot& sl = s->slots[k];
        sl.state = FILLING;
        sl.beam = beam;
        sl.seq = seq;
        sample0 = b.next_sample;
        sl.sample0 = sample0;
        sl.t_push = t_arrive;
        b.started = true;
        b.next_seq = seq + 1;
        b.next_sample = sample0 + s->hop;
        if (!s->have_first) {
            s->t_first = t_arrive;
            s->have_first = true;
        }
        s->inflight++;
        s->max_inflight = std::max(s->max_inflight, s->inflight);
    }
    Slot& sl = s->slots[k];
    BeamState& b = s->beams[beam];
    const size_t W = (size_t)s->window, D = (size_t)s->dmax, H = (size_t)s->hop;
    cudaStream_t st = sl.stream;
    int rc = AF_OK;
    cudaError_t e;
    if (first) {
        e = cudaMemcpy2DAsync(sl.d_in, W, h_data, (size_t)pitch, W, s->nchan, cudaMemcpyHostToDevice, st);
    } else {
        e = cudaStreamWaitEvent(st, b.overlap_ready, 0);
        if (e == cudaSuccess && D > 0)
            e = cudaMemcpy2DAsync(sl.d_in, W, b.d_overlap, D, D, s->nchan, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(sl.d_in + D, W, h_data, (size_t)pitch, H, s->nchan, cudaMemcpyHostToDevice, st);
    }
    // the next window of this beam starts with this window's last Dmax samples
    if (e == cudaSuccess && D > 0)
        e = cudaMemcpy2DAsync(b.d_overlap, D, sl.d_in + H, W, D, s->nchan, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(b.overlap_ready, st);
    if (e == cudaSuccess) e = cudaEventRecord(sl.input_ready, st);
    // the caller may reuse h_data when push returns
    if (e == cudaSuccess) e = cudaEventSynchronize(sl.input_ready);
    if (e != cudaSuccess) rc = af_cuda_check(e, "af_stream_push: copy");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (rc) {
            sl.state = FREE;
            s->inflight--;
            s->error = rc;
            s->error_msg = af_last_error();
            return rc;
        }
        sl.state = READY;
        s->ready.push_back(k);
    }
    s->cv_ready.notify_one();
    return AF_OK;
} catch (...) {
    return af_host_exception("af_stream_push");
}

extern "C" int af_stream_poll(af_stream_t s, af_stream_result_t* out, int timeout_ms)
try {
    if (!s || !out) return af_set_error(AF_EINVAL, "af_stream_poll: NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && !s->error) {
        if (timeout_ms <= 0) return AF_EAGAIN;
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !s->done.empty() || s->error; });
    }
    if (s->done.empty()) {
        if (s->error) return af_set_error(s->error, "af_stream_poll: the engine failed: %s", s->error_msg.c_str());
        return AF_EAGAIN;
    }
    const int k = s->done.front();
    s->done.pop_front();
    Slot& sl = s->slots[k];
    sl.state = HELD;
    const double lat = std::chrono::duration<double, std::milli>(sl.t_done - sl.t_push).count();
    s->lat_ms.push_back(lat);
    s->windows_done++;
    s->t_last = sl.t_done;
    s->inflight--;
    out->beam = sl.beam;
    out->seq = sl.seq;
    out->sample0 = sl.sample0;
    out->slot = k;
    out->total = *sl.h_count;
    out->count = std::min(*sl.h_count, s->cap);
    out->cands = sl.h_cands;
    out->latency_ms = lat;
    out->status = *sl.h_count > s->cap ? AF_EOVERFLOW : AF_OK;
    lk.unlock();
    if (out->count > 1)
        std::sort(sl.h_cands, sl.h_cands + out->count, [](const af_cand_t& p, const af_cand_t& q) {
            return p.dm_idx != q.dm_idx ? p.dm_idx < q.dm_idx : p.t < q.t;
        });
    int flag = 0;
    if (cudaMemcpy(&flag, s->d_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && flag) {
        cudaMemset(s->d_err, 0, sizeof(int));
        out->status = AF_ETIMEOUT;
    }
    return AF_OK;
} catch (...) {
    return af_host_exception("af_stream_poll");
}

extern "C" int af_stream_release(af_stream_t s, int32_t slot)
try {
    if (!s || slot < 0 || slot >= (int)s->slots.size()) return af_set_error(AF_EINVAL, "af_stream_release: bad slot");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->slots[slot].state != HELD) return af_set_error(AF_EINVAL, "af_stream_release: slot %d not held", slot);
        s->slots[slot].state = FREE;
    }
    s->cv_free.notify_all();
    return AF_OK;
} catch (...) {
    return af_host_exception("af_stream_release");
}

extern "C" int af_stream_result_plane(af_stream_t s, int32_t slot, int32_t** d_plane, float** d_snr, int64_t* nout)
try {
    if (!s || slot < 0 || slot >= (int)s->slots.size()) return af_set_error(AF_EINVAL, "af_stream_result_plane: bad slot");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->slots[slot].state != HELD) return af_set_error(AF_EINVAL, "af_stream_result_plane: slot not held");
    if (d_plane) *d_plane = s->slots[slot].d_plane;
    if (d_snr) *d_snr = s->slots[slot].d_snr;
    if (nout) *nout = s->hop;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_stream_result_plane");
}

extern "C" int af_stream_classify(af_stream_t s, int32_t slot, af_model_t model, const af_cand_t* h_cands, int32_t n,
                                  float* h_prob)
try {
    if (!s || !model || slot < 0 || slot >= (int)s->slots.size() || n < 0 || n > s->cap ||
        (n > 0 && (!h_cands || !h_prob)))
        return af_set_error(AF_EINVAL, "af_stream_classify: bad arguments (n must be <= the engine's cap)");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->slots[slot].state != HELD) return af_set_error(AF_EINVAL, "af_stream_classify: slot %d not held", slot);
    }
    if (n == 0) return AF_OK;
    Slot& sl = s->slots[slot];
    cudaStream_t cs = s->cstream;
    AF_CUDA(cudaMemcpyAsync(s->d_ccands, h_cands, (size_t)n * sizeof(af_cand_t), cudaMemcpyHostToDevice, cs));
    if (int rc = af_classify(model, s->plan, sl.d_in, s->window, sl.d_plane, s->hop, s->d_ccands, n, s->d_cprob, cs))
        return rc;
    AF_CUDA(cudaMemcpyAsync(h_prob, s->d_cprob, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, cs));
    AF_CUDA(cudaStreamSynchronize(cs));
    return AF_OK;
} catch (...) {
    return af_host_exception("af_stream_classify");
}

extern "C" int af_stream_cluster(af_stream_t s, af_cand_t* h_cands, int32_t n, af_cand_t* h_out, int32_t* n_out)
try {
    if (!s) return af_set_error(AF_EINVAL, "af_stream_cluster: NULL stream");
    return af_cluster(s->plan, h_cands, n, 20.0, 0.2, h_out, n_out);
} catch (...) {
    return af_host_exception("af_stream_cluster");
}

extern "C" int af_stream_info(af_stream_t s, int64_t* hop, int64_t* dmax, int* nslots)
try {
    if (!s) return af_set_error(AF_EINVAL, "af_stream_info: NULL stream");
    if (hop) *hop = s->hop;
    if (dmax) *dmax = s->dmax;
    if (nslots) *nslots = (int)s->slots.size();
    return AF_OK;
} catch (...) {
    return af_host_exception("af_stream_info");
}

extern "C" int af_stream_stats(af_stream_t s, af_stream_stats_t* st)
try {
    if (!s || !st) return af_set_error(AF_EINVAL, "af_stream_stats: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(st, 0, sizeof *st);
    st->windows = s->windows_done;
    st->launches = s->launches;
    st->max_inflight = s->max_inflight;
    st->slots = (int)s->slots.size();
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (v.size() - 1) + 0.5))]; };
        st->p50_ms = q(0.50);
        st->p99_ms = q(0.99);
        st->max_ms = v.back();
    }
    if (s->have_first && s->windows_done > 0) {
        st->wall_s = std::chrono::duration<double>(s->t_last - s->t_first).count();
        const double work = (double)s->windows_done * s->ndm * s->nchan * (double)s->hop;
        st->work = work;
        st->rate = st->wall_s > 0 ? work / st->wall_s : 0.0;
    }
    return AF_OK;
} catch (...) {
    return af_host_exception("af_stream_stats");
}

extern "C" int af_stream_snapshot(af_stream_t s, int beam, uint8_t* h_overlap, int64_t* next_seq,
                                  int64_t* next_sample)
try {
    if (!s || beam < 0 || beam >= s->nbeams) return af_set_error(AF_EINVAL, "af_stream_snapshot: bad beam");
    BeamState& b = s->beams[beam];
    AF_CUDA(cudaEventSynchronize(b.overlap_ready));
    if (h_overlap && s->dmax > 0)
        AF_CUDA(cudaMemcpy(h_overlap, b.d_overlap, (size_t)s->nchan * s->dmax, cudaMemcpyDeviceToHost));
    std::lock_guard<std::mutex> lk(s->mu);
    if (next_seq) *next_seq = b.next_seq;
    if (next_sample) *next_sample = b.next_sample;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_stream_snapshot");
}

extern "C" int af_stream_restore(af_stream_t s, int beam, const uint8_t* h_overlap, int64_t next_seq,
                                 int64_t next_sample)
try {
    if (!s || beam < 0 || beam >= s->nbeams || (!h_overlap && s->dmax > 0) || next_seq < 1 || next_sample < 0)
        return af_set_error(AF_EINVAL, "af_stream_restore: bad arguments");
    BeamState& b = s->beams[beam];
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (b.started) return af_set_error(AF_EINVAL, "af_stream_restore: beam %d already streaming", beam);
    }
    if (s->dmax > 0)
        AF_CUDA(cudaMemcpy(b.d_overlap, h_overlap, (size_t)s->nchan * s->dmax, cudaMemcpyHostToDevice));
    AF_CUDA(cudaEventRecord(b.overlap_ready, 0));
    AF_CUDA(cudaEventSynchronize(b.overlap_ready));
    std::lock_guard<std::mutex> lk(s->mu);
    b.started = true;
    b.next_seq = next_seq;
    b.next_sample = next_sample;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_stream_restore");
}

extern "C" int af_stream_close(af_stream_t s)
try {
    free_stream(s);
    return AF_OK;
} catch (...) {
    return af_host_exception("af_stream_close");
}
