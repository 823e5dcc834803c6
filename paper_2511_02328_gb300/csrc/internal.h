// internal.h -- shared declarations of the afgb library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "afgb.h"

// ---------------------------------------------------------------- errors
int af_set_error(int code, const char* fmt, ...);
int af_cuda_check(cudaError_t e, const char* what);
// Status for a C++ exception that reached an entry point (call it only inside a
// catch handler): AF_ENOMEM for std::bad_alloc, else AF_EINVAL, with a message.
// Every extern "C" int entry point is a function-try-block ending in it, so no
// exception crosses the C ABI.
int af_host_exception(const char* who);
#define AF_CUDA(call)                                                  \
    do {                                                               \
        cudaError_t _e = (call);                                       \
        if (_e != cudaSuccess) return af_cuda_check(_e, #call);        \
    } while (0)

// ---------------------------------------------------------------- widths
// Boxcar widths passed to kernels by value.
struct af_widths_t {
    int32_t w[AF_MAX_WIDTHS];
    int32_t n;
    int32_t small;  // every window sum (hence B - q) is below 2^31: 32-bit difference
};

// Per-row, per-width S/N constants:  snr = float(B - q) * k - c  with
// q = floor(w*S/nout), k = 1/(sigma*sqrt(w)), c = ((w*S - q*nout)/nout) * k.
struct af_rowconst_t {
    int64_t q;
    float k;
    float c;
};

// ---------------------------------------------------------------- tile tables
// Device tables of the tile dedispersion kernel for one delay table and block
// shape (nw DM rows per block, m 128-output groups per lane).
struct af_tile_tables {
    int nw = 0, m = 0;
    int32_t* d_dsort = nullptr;    // [ndm_pad][nchan] delays in ascending-DM order
    int32_t* d_perm = nullptr;     // [ndm_pad] plane row of each sorted DM (-1: padding)
    int32_t* d_dminblk = nullptr;  // [nblk][nchan] smallest delay per block and channel
    int ndm_pad = 0, nblk = 0, spread = 0, rw = 0;
    bool fits = false;             // the channel window fits in shared memory with the 4-deep ring
    int ns1 = 0;                   // ring depth of the single-plan kernel: 4, else 3 or 2 (coarse DM
                                   // grids), 0 if none fits
};
// Raises a kernel's dynamic shared-memory limit to at least `bytes` (the
// attribute belongs to the kernel, not to a plan: it only ever grows).
int af_ensure_smem(const void* kernel, size_t bytes);

int af_tile_tables_build(const int32_t* delays, const double* dms, int ndm, int nchan, int nw, int m, int device,
                         af_tile_tables* t, std::vector<int32_t>* h_dsort = nullptr,
                         std::vector<int32_t>* h_dmin = nullptr);
void af_tile_tables_free(af_tile_tables* t);
size_t af_tile_smem(int nw, int rw, int ns = 4);

// ---------------------------------------------------------------- subband
// Device side of a two-stage subband plan (Sec. 2.3): stage-1 tile tables
// over the coarse DMs (staggered delays), the stagger and partition tables,
// the residual shifts and the stage-1 scratch I [ncoarse][nsub][ipitch].
struct af_sb_device {
    af_tile_tables tile;           // stage-1 tables (rows = coarse DMs)
    int32_t* d_stag = nullptr;     // [ndm_pad][nsub]
    int32_t* d_first = nullptr;    // [nsub+1]
    int32_t* d_r = nullptr;        // [ndm][nsub] residual shifts
    void* d_I = nullptr;           // stage-1 scratch
    bool i16 = false;              // I holds uint16 (every subband <= 257 channels)
    int64_t ipitch = 0;            // elements per I row
    int32_t maxstag = 0;           // largest stagger
    int cps = 0;                   // 32-channel chunks per subband
};

// ---------------------------------------------------------------- group rows
// Arguments of one group-row stage-2 launch (a plan's time block).
struct af_pair_args {
    const uint16_t* PS;      // rows of the time block
    const int2* chunks;      // per chunk: {row slots, first slot}
    const int32_t* chkoff;   // [nblk + 1] first chunk of each block
    const int* tabs;         // per chunk: NW x TABW ints, every consumer warp's table for its ring stage
    const int2* srec;        // per slot: {window bytes, byte offset inside its stage}
    const int64_t* soff;     // per slot: element offset of its window in PS for the block's first tile
    const int32_t* perm;     // [ndm_pad] plane row, -1 = padding
    int stage_bytes;         // bytes of one ring stage's windows
    int flush;               // rows between folds: flush * 255 * G < 2^16
    unsigned nblk;
    int64_t T0;              // first output of the time block (a multiple of 8)
    int64_t tend;            // outputs t < tend are written
    int64_t nout;
    int32_t* Y;
    af_rowstats_t* stats;
    int* err;
};

// Single-plan dedispersion through channel-group rows (pairs.cu): host tables
// (built once per plan), device tables, and the row buffer of one time block.
struct af_pair_tables {
    bool ok = false;               // the plan can use this path
    int G = 2;                     // channels per group (2, 3 or 4)
    int np = 0, nrows = 0, rwe = 0, maxdr = 0;   // np = groups
    double rows_per_pair = 0;      // rows copied per pair and DM block (mean)
    size_t budget = 0;             // bytes the row buffer may take (AFGB_PAIR_BUDGET_MB at plan creation)
    int shape = 0;                 // ring depth of the row kernel (2 to 4 stages)
    int stage_bytes = 0;           // bytes of one ring stage (windows packed back to back)
    af_tile_tables tt;             // DM order and block minima for this block shape
    double copy_per_tile = 0;      // bytes of row windows copied per time tile (all DM blocks)
    std::vector<int32_t> h_rb, h_ub, h_rB, h_rspan, h_srow, h_scpart;
    int32_t* d_rdelta = nullptr;   // [nrows][G-1] relative delays of each row
    int2* d_gdr = nullptr;         // [groups][G-1] smallest and largest relative delay
    int2* d_chunks = nullptr;      // per chunk: row slots, first slot
    int32_t* d_chkoff = nullptr;   // [nblk + 1]
    int* d_tabs = nullptr;         // per chunk: every consumer warp's table
    int2* d_srec = nullptr;        // per slot: window bytes, byte offset inside its ring stage
    uint16_t* d_ps = nullptr;      // row buffer
    size_t ps_bytes = 0;
    bool ps_owned = true;          // false: a buffer shared by a batch's plans
    // Row-buffer layouts made by the reservation calls: 0 for af_dedisperse
    // (the longest time block the budget allows), 1 for af_search (at least
    // eight blocks, so that the input copy overlaps the work).
    struct Layout {
        int64_t L = 0, maxlen = 0;     // outputs per time block, longest row
        int4* d_pinfo = nullptr;       // [np] first row, rows, range start ub, range length
        int2* d_rinfo = nullptr;       // [nrows] row start - ub, row length (rows of a group by start)
        int* d_gmax = nullptr;         // [np] longest row of each group
        int64_t* d_rowoff = nullptr;   // [nrows] element offset in the row buffer
        int64_t* d_soff = nullptr;     // per slot: window offset for a time block's first tile
    } lay[2];
    // optional stage timing of af_dedisperse calls (af_dedisperse_timing):
    // events [call % ncalls][block][3] = before stage 1, between, after stage 2
    std::vector<cudaEvent_t> tev;
    int tcalls = 0, tblocks = 0, tnext = 0;
    std::vector<int> tnb;              // blocks recorded per call slot
    std::vector<int64_t> trowbytes;    // row-buffer bytes written per call slot
    std::vector<int64_t> tcopybytes;   // row-window bytes copied into shared memory per call slot
};
int af_pairs_build(af_plan_t p);
void af_pairs_free(af_pair_tables* T);
int64_t af_pairs_block(af_plan_t p, int64_t nout);
int af_pairs_reserve(af_plan_t p, int64_t nout, bool search, bool allow_larger = true,
                     size_t max_bytes = SIZE_MAX);
int af_pairs_pick(af_plan_t p, int64_t nout, bool allow_larger, size_t max_bytes, int64_t* L);
size_t af_pairs_workspace(af_plan_t p, int64_t nout);  // row-buffer bytes a reservation would allocate
// Stage 1 alone (the rows of time block T0 of layout `layout`), the stage-2
// arguments of that block (and its item count: tiles x DM blocks), the
// stage-2 shared memory of a ring of ns stages, the plan's ring depth, and
// one persistent stage-2 launch over many plans' blocks (jobs in device
// memory, first[j] = items before job j, first[njobs] = total).
// Lb = the block's length (a multiple of the tile, at most the layout's; 0 = the layout's); T0 a multiple of the tile.
int af_launch_pairs_rows(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int layout, int64_t T0, cudaStream_t s,
                         int64_t Lb = 0);
int af_pairs_block_args(af_plan_t p, int64_t nout, int layout, int64_t T0, int32_t* d_plane, af_rowstats_t* d_stats,
                        af_pair_args* out, long long* items, int64_t Lb = 0);
size_t af_pairs_stage2_smem(af_plan_t p, int ns);
int af_pairs_ring(af_plan_t p);
int af_launch_pairs_persistent(int ns, size_t smem, int grid, const af_pair_args* d_jobs, const long long* d_first,
                               int njobs, long long total, unsigned long long* d_counter, cudaStream_t s);
int af_launch_pairs(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int64_t nout, int32_t* d_plane,
                    af_rowstats_t* d_stats, cudaStream_t s);
// Stage 1 + stage 2 of the time block starting at T0 (a multiple of the
// layout's block length; row sums accumulate, the caller clears them once).
int af_launch_pairs_block(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int64_t nout, int32_t* d_plane,
                          af_rowstats_t* d_stats, cudaStream_t s, int layout, int64_t T0,
                          cudaEvent_t* mid = nullptr, int64_t Lb = 0);
// The time blocks af_search runs on nout outputs, in tiles: the first small
// (its input, outputs + Dmax, is copied before any work), each next one six
// times the previous (its input arrives while the previous one runs), at most
// cap_tiles each.
std::vector<int64_t> af_search_block_tiles(int64_t nout, int64_t cap_tiles);
int af_pair_tile_outputs();
int af_pair_ring_depth(int shape);
// Row-buffer bytes of a full-length single time block, and the use of a row
// buffer owned by someone else (a batch's plans run one after another on one).
size_t af_pairs_bytes(af_plan_t p, int64_t nout);
size_t af_pairs_reserved_bytes(af_plan_t p, int64_t nout);  // what af_pairs_reserve would allocate
int af_pairs_attach(af_plan_t p, uint16_t* buf, size_t bytes, int64_t nout);
bool af_dedisp_uses_pairs(af_plan_t p, int64_t nout);

// ---------------------------------------------------------------- plan
struct af_plan_s {
    int nchan = 0;
    int ndm = 0;
    double f_lo = 0, f_hi = 0, tsamp = 0;
    int32_t dmax = 0;
    int device = 0;
    std::vector<double> dms;
    std::vector<int32_t> delays;           // [ndm][nchan]
    int num_sms = 0;

    // device copies and scratch (owned)
    int32_t* d_delays = nullptr;           // [ndm][nchan]
    af_tile_tables tile;                   // tables of the tile dedispersion kernel
    int* d_err = nullptr;                  // device error flag (bounded waits that ran out)
    bool force_simple = false;             // use the fallback kernel (AFGB_DEDISP_KERNEL=simple)
    bool force_brute = false;              // subband plans: brute-force tile kernel on the
                                           // effective delays (AFGB_DEDISP_KERNEL=brute)
    bool force_tile = false;               // byte tile kernel even where group rows apply
                                           // (AFGB_DEDISP_KERNEL=tile)
    bool force_pairs = false;              // group rows wherever they apply, without the cost
                                           // comparison (AFGB_DEDISP_KERNEL=pairs)
    int force_group = 0;                   // 2, 3 or 4: only that group size (AFGB_PAIR_GROUP)
    af_pair_tables pairs;                  // group-row path of brute-force plans (the one in use)
    af_pair_tables alt[2];                 // the other group sizes (3, 4), until a reservation picks

    // two-stage subband dedispersion (sb_nsub > 0); `delays` then holds the
    // effective table D[j(m)][c] + R[m][s(c)]
    int sb_n0 = 0, sb_nsub = 0, sb_ncoarse = 0, sb_mode = 0;
    int64_t sb_L = 0;                      // stage-2 outputs per time block
    int32_t sb_rmax = 0;                   // largest residual shift
    std::vector<int32_t> sb_first;         // [nsub+1]
    std::vector<double> sb_F;              // [nsub] representative frequencies
    std::vector<double> sb_cdms;           // [ncoarse] coarse DMs
    std::vector<int32_t> sb_dc;            // [ncoarse][nchan] coarse delays
    std::vector<int32_t> sb_r;             // [ndm][nsub] residual shifts
    af_sb_device sb;
    af_rowstats_t* d_stats = nullptr;      // [ndm] scratch
    af_rowconst_t* d_rowconst = nullptr;   // [ndm][AF_MAX_WIDTHS] scratch

    // reserved workspace of af_search
    int64_t ws_nsamp = 0;
    int32_t ws_cap = 0;
    uint8_t* ws_in = nullptr;
    int32_t* ws_plane = nullptr;
    float* ws_snr = nullptr;
    uint8_t* ws_bw = nullptr;
    af_cand_t* ws_cands = nullptr;
    int32_t* ws_count = nullptr;
    int32_t* ws_host = nullptr;            // pinned: count, error flag, 2 pad words, then ws_stage candidates
    int32_t ws_stage = 0;                  // candidates copied back with the count (one wait per search)
    cudaStream_t ws_copy = nullptr;        // input copies of af_search, overlapped with dedispersion
    cudaEvent_t ws_ev[4] = {};             // one per copied time segment
    // optional phase timing of af_search (af_search_timing): events on the
    // caller's stream at the start, when the first block may run (its input
    // is in), after the dedispersion, after S/N + candidates
    bool ws_timing = false;
    std::vector<int32_t> ws_band;          // af_search's input copies: channel bands [ws_band[j], ws_band[j+1])
    std::vector<int32_t> ws_band_dmax;     // ... and each band's largest delay over every DM
    cudaEvent_t ws_tev[4] = {};
};

int af_check_plan(af_plan_t p);
int af_check_widths(af_plan_t p, const int32_t* widths, int nw, int64_t nout, af_widths_t* out);
// The same checks for planes summed over `nchan` channels of 8-bit data (no
// plan needed); sets .small when every window sum is below 2^31.
int af_check_widths_nchan(int nchan, const int32_t* widths, int nw, int64_t nout, af_widths_t* out);

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `s` and return AF_OK or AF_ECUDA (launch error).
int af_launch_dedisperse(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int64_t nout,
                         int32_t* d_plane, af_rowstats_t* d_stats, cudaStream_t s);
int af_launch_rowstats(const int32_t* d_plane, int ndm, int64_t nout, af_rowstats_t* d_stats,
                       cudaStream_t s);
// Brute-force tile kernel on output tiles [tile_begin, tile_end) only (row sums
// accumulate; the caller clears them once), its tile length, and whether a plan
// uses it.
int af_launch_dedisperse_tiles(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int64_t nout, int32_t* d_plane,
                               af_rowstats_t* d_stats, cudaStream_t s, unsigned tile_begin, unsigned tile_end);
int af_dedisp_tile_outputs();
bool af_dedisp_uses_tiles(af_plan_t p);
int af_launch_boxcar(const int32_t* d_plane, int ndm, int64_t nout, const af_rowstats_t* d_stats,
                     const af_widths_t& w, af_rowconst_t* d_rowconst, float* d_best_snr,
                     uint8_t* d_best_w, cudaStream_t s);
int af_launch_candidates(const float* d_best_snr, const uint8_t* d_best_w, int ndm, int64_t nout,
                         const af_widths_t& w, float thresh, int64_t sample0, af_cand_t* d_out,
                         int32_t cap, int32_t* d_count, cudaStream_t s);
int af_prepare_dedisp_tables(af_plan_t p);
int af_launch_row_robust(const int32_t* d_plane, int ndm, int64_t nout, af_robust_t* d_robust, cudaStream_t s);
int af_launch_boxcar_robust(const int32_t* d_plane, int ndm, int64_t nout, const af_robust_t* d_robust,
                            const af_widths_t& w, af_rowconst_t* d_rowconst, float* d_best_snr, uint8_t* d_best_w,
                            cudaStream_t s);
// Subband plans: builds the device tables and the scratch (af_plan_subband);
// frees them (plan destruction); launches stage 1 + stage 2 per time block.
int af_sb_prepare(af_plan_t p);
void af_sb_free(af_plan_t p);
int af_launch_subband(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int64_t nout, int32_t* d_plane,
                      af_rowstats_t* d_stats, cudaStream_t s);
