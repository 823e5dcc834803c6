/*
 * afgb.h -- C ABI of the GB300 (sm_103a) single-pulse search library.
 *
 * The library implements the hot path of the single-pulse search of
 * ASTROFLOW (arXiv 2511.02328): exact brute-force incoherent dedispersion of
 * 8-bit filterbank data into an int32 DM-time plane (Sec. 2.3), boxcar
 * matched filtering with S/N normalisation (step (iii) of the workflow in
 * Sec. 1) and thresholding into a candidate list (Sec. 2), with the
 * true-positive clustering rule of Sec. 4.2.
 *
 * Conventions shared by every call:
 *  - Every call returns an int status: AF_OK (0) or one of the AF_E* codes.
 *    af_last_error() returns a thread-local message for the last failure.
 *  - Errors, unless a call's own comment adds to them: AF_EINVAL for a NULL
 *    handle, a NULL required pointer or a size outside its stated range
 *    (checked before any work is enqueued); AF_ECUDA when a CUDA call or a
 *    launch fails; AF_ENOMEM when an allocation fails (only the calls that
 *    create, reserve, build or open allocate device or pinned memory; the
 *    *_timing calls create CUDA events).  A call rejected for its arguments
 *    has enqueued nothing and changed nothing.
 *  - Pointers named d_* are DEVICE pointers owned by the caller (for example
 *    torch tensors); pointers named h_* or host_* are host pointers owned by
 *    the caller.  The library never frees caller memory.
 *  - Handles (af_plan_t, af_batch_t, af_stream_t, af_model_t) are owned by
 *    the library and freed by the matching *_destroy call.
 *  - Calls that take `void* stream` (a cudaStream_t; NULL = legacy default
 *    stream) only ENQUEUE work on that stream and return at once; results are
 *    valid after the stream is synchronised.  Argument errors are reported
 *    synchronously, before anything is enqueued.
 *  - No call that launches work allocates device memory.  Scratch lives in the
 *    plan (sized at af_plan time) or in a reservation made by an explicit
 *    *_reserve call.
 *  - Filterbank data are uint8, channel-major: x[c * nsamp + t].
 *  - A plan is not thread-safe: calls on the same plan must not overlap in
 *    host threads, and work enqueued on different streams with the same plan
 *    shares the plan's scratch (serialise such streams).
 */
#ifndef AFGB_H
#define AFGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define AF_OK        0
#define AF_EINVAL    1  /* invalid argument (sizes, pointers, ordering)      */
#define AF_ENOMEM    2  /* device or host allocation failed                  */
#define AF_ENOBUFS   3  /* request exceeds a reservation or an HBM budget     */
#define AF_ECUDA     4  /* a CUDA runtime call failed; see af_last_error()   */
#define AF_ETIMEOUT  5  /* a bounded device or host wait ran out             */
#define AF_EOVERFLOW 6  /* more candidates than capacity; count is the total */
#define AF_EAGAIN    7  /* nothing ready yet (polling calls)                 */

#define AF_MAX_WIDTHS 32 /* maximum number of boxcar widths per call         */
#define AF_NO_WIDTH 0xFF /* best-width index where no width fits (tail)      */
#define AF_NOALLOC_MAX_ROWS 4096 /* row limit of af_boxcar_snr_noalloc       */

typedef struct af_plan_s* af_plan_t;
typedef struct af_model_s* af_model_t;  /* the candidate classifier, see below */

/* Per-DM-row sums of the plane: sum = sum_t Y[d][t], sumsq = sum_t Y[d][t]^2
 * over the row's nout samples (exact 64-bit integers). */
typedef struct {
    int64_t sum;
    int64_t sumsq;
} af_rowstats_t;

/* One candidate: DM row, output time index t of the window's leading edge
 * (arrival time at f_ref, the top of the band), boxcar width in samples,
 * S/N, and abs_sample = sample0 + t (sample0 is given by the caller, e.g. the
 * first sample of a streamed chunk).  TOA in seconds = abs_sample * tsamp. */
typedef struct {
    int32_t dm_idx;
    int32_t t;
    int32_t width;
    float snr;
    int64_t abs_sample;
} af_cand_t;

/* Thread-local message describing the last failing call ("" if none). */
const char* af_last_error(void);

/* Library version string. */
const char* af_version(void);

/* ---- plan: channel frequencies and the integer delay table ------------- *
 * Builds the delay table of Eq. (coarse_delay), Sec. 2.3, for an explicit DM
 * list:
 *     D[d][c] = round( K_DM * dm_list[d] / tsamp * (1/f_c^2 - 1/f_ref^2) )
 * with K_DM = 4.148808e3 s MHz^2 pc^-1 cm^3 (Eq. KDM; the paper prints the
 * unit as ms, the value is in seconds with f in MHz), f_c the CENTRE of
 * channel c, f_c = f_lo + (c + 0.5) * (f_hi - f_lo) / nchan, f_ref =
 * max(f_lo, f_hi) (top of the band), round = half away from zero, evaluated
 * in IEEE double as a = (K*dm)/tsamp, b = 1/(fc*fc) - 1/(fr*fr), D = llround(a*b)
 * with no fused multiply-add.
 *  nchan   number of channels (1 .. 65536)
 *  f_lo    band edge on channel 0's side, MHz (> 0)
 *  f_hi    band edge on channel nchan-1's side, MHz (> 0, != f_lo); f_hi < f_lo
 *          means channel 0 is the highest frequency
 *  tsamp   sampling interval, seconds (> 0)
 *  dm_list host array of ndm trial DMs, pc cm^-3, each >= 0 and finite; any
 *          order (rows of the plane follow this order)
 *  ndm     1 .. 1<<20
 * The plan copies everything it needs, uploads the table to the current
 * device and allocates its scratch there (AF_ENOMEM / AF_ECUDA on failure).
 * AF_EINVAL if an argument is out of range or a delay exceeds int32. */
int af_plan(af_plan_t* out, int nchan, double f_lo, double f_hi, double tsamp,
            const double* dm_list, int ndm);

/* Frees the plan and everything it allocated (NULL is accepted). */
int af_plan_destroy(af_plan_t plan);

/* Copies the delay table to host_out ([ndm][nchan] int32, may be NULL) and
 * the largest delay Dmax to *dmax (may be NULL). */
int af_plan_delays(af_plan_t plan, int32_t* host_out, int32_t* dmax);

/* Plan dimensions (any output pointer may be NULL). */
int af_plan_info(af_plan_t plan, int* nchan, int* ndm, int32_t* dmax, double* tsamp);

/* Which kernel af_dedisperse runs for this plan (any output may be NULL):
 *  path    AF_PATH_SIMPLE (one thread per output, every delay read from the
 *          table), AF_PATH_TILE (the shared-memory tile kernel over channels),
 *          AF_PATH_SUBBAND (the two stages of Sec. 2.3) or AF_PATH_PAIRS (the
 *          same exact sum over channel-group rows: the channels of a group
 *          (2, 3 or 4 adjacent channels) added once per distinct tuple of
 *          relative delays, then a tile kernel over group rows; reported once
 *          af_dedisperse_reserve or af_search_reserve has reserved the row
 *          buffer);
 *  ring    depth of the kernel's shared-memory ring (4; 3 or 2 when a coarse
 *          DM grid widens each channel's window; 2 to 4 for group rows), 0 on
 *          the simple path;
 *  spread  largest delay difference between DMs of one block of the kernel,
 *          in samples (what sets the window width);
 *  group   channels per row: 2, 3 or 4 on the group-row path, else 1.
 * AFGB_DEDISP_KERNEL=tile|simple|pairs in the environment at plan creation
 * forces the channel tile kernel, the simple kernel, or group rows wherever
 * they apply (without the cost comparison); AFGB_PAIR_GROUP=2|3|4 fixes the
 * group size.  Read-only; no device work.  Not a step of the paper's method. */
#define AF_PATH_SIMPLE 0
#define AF_PATH_TILE 1
#define AF_PATH_SUBBAND 2
#define AF_PATH_PAIRS 3
int af_plan_kernel(af_plan_t plan, int* path, int* ring, int32_t* spread, int* group);

/* Reads and clears the plan's device error flag, which a kernel of this plan
 * sets when one of its bounded waits (for an asynchronous copy) ran out and it
 * abandoned its work; returns AF_ETIMEOUT if the flag was set, else AF_OK.
 * Blocks until all work on the device has finished. */
int af_plan_check(af_plan_t plan);

/* Output length for nsamp input samples: nout = nsamp - Dmax (reading of the
 * paper's truncation by the DM delay, Sec. 3).  AF_EINVAL if nout <= 0. */
int af_plan_nout(af_plan_t plan, int64_t nsamp, int64_t* nout);

/* ---- channel-range plan: the multi-band search, Sec. 2.2 ---------------- *
 * A plan for the channels [c0, c1) of a band of nchan channels between f_lo
 * and f_hi.  Channel centres and f_ref are those of the WHOLE band, so its
 * delay table is columns [c0, c1) of the whole band's table and its
 * candidates' TOAs refer to the whole band's top edge.  Its input is the
 * [c1 - c0][nsamp] block of rows starting at channel c0 (d_in + c0 * nsamp of
 * the whole band's array; af_dedisperse requires that address to be 16-byte
 * aligned).  The paper's F+L+H search (its configurations A2/A3: F = 1000-1500,
 * L = 1000-1250, H = 1250-1500 MHz) is three such plans, [0, nchan),
 * [0, nchan/2) and [nchan/2, nchan), searched separately; the union of their
 * candidates (same dm_list and tsamp, so the same dm_idx and abs_sample units)
 * is merged by af_cluster.  The planes add up: Y_F = Y_L + Y_H on the first
 * nout_F outputs.  Other arguments and errors as af_plan; AF_EINVAL unless
 * 0 <= c0 < c1 <= nchan. */
int af_plan_channels(af_plan_t* out, int nchan, double f_lo, double f_hi, double tsamp,
                     const double* dm_list, int ndm, int c0, int c1);

/* ---- square-law time downsampling, Sec. 2.2 ------------------------------ *
 * For every channel and bin k of D consecutive samples (the last bin holds the
 * remaining nsamp - (nout-1)*D; nout = ceil(nsamp/D)), with S the bin's sum and
 * N its sample count:
 *     out = min( V * sqrt(S) / sqrt(N * V), V ) = min( sqrt(V*S/N), V ),  V = 255,
 * rounded to nearest with halves up, exactly: floor((isqrt(floor(4*V*S/N)) + 1) / 2).
 *  d_in   uint8 [nchan][nsamp] (channel-major)
 *  D      1 .. 32768
 *  d_out  uint8 [nchan][ceil(nsamp/D)] (caller-owned)
 * The output is searched with a plan whose tsamp is D * tsamp (the paper's
 * t_samp on the downsampled grid, Eq. coarse_delay).  Enqueued on `stream`. */
int af_downsample(const uint8_t* d_in, int nchan, int64_t nsamp, int D, uint8_t* d_out, void* stream);

/* ---- zero-DM filter, Sec. 2.1 ------------------------------------------- *
 * Removes the DM = 0 time series (the paper's zero-DM filter, named among its
 * RFI steps in Sec. 2.1 and as the remedy for impulsive broadband RFI in
 * Sec. 4.4; the formula is a reading): for every time sample t, with the mean
 * over channels rounded half up, q[t] = floor((2 * sum_c X[c][t] + nchan) / (2 * nchan)),
 *     out[c][t] = min(255, max(0, X[c][t] - q[t] + 128)),
 * i.e. re-centred on mid-scale so that the result stays 8-bit.
 *  d_in, d_out uint8 [nchan][nsamp] (d_out == d_in filters in place), nchan <= 65536.
 * Enqueued on `stream`. */
int af_zerodm(const uint8_t* d_in, int nchan, int64_t nsamp, uint8_t* d_out, void* stream);

/* ---- subband plan: two-stage subband dedispersion, Sec. 2.3 ------------ *
 * The paper's own dedispersion scheme (Eqs. stage1, residual, stage2).  The
 * channels are split into nsub contiguous subbands, subband s = channels
 * [floor(s*nchan/nsub), floor((s+1)*nchan/nsub)), each with a representative
 * frequency F_s; the fine DM list is grouped n0 at a time, j(m) = m / n0, with
 * coarse DM_j = dm_list[j*n0] (DM_low + j*n0*dDM for an evenly spaced list):
 *   stage 1  I(j,s,u) = sum_{c in s} X[c][u + D[j][c]]   D: Eq. (coarse_delay) at DM_j
 *   stage 2  Y[m][v]  = sum_s I(j(m), s, v + R[m][s])
 *   R[m][s] = round(K*(dm_list[m] - DM_j(m))/tsamp * (1/F_s^2 - 1/f_ref^2))   Eq. (residual)
 * with the channel centres, f_ref and rounding of af_plan.  The plane is the
 * brute-force sum with the EFFECTIVE delay table
 *     Deff[m][c] = D[j(m)][c] + R[m][s(c)],
 * so af_plan_delays returns Deff, Dmax = max Deff, nout = nsamp - Dmax, and
 * af_dedisperse, af_boxcar_snr, af_candidates, af_search, af_cutouts and
 * af_classify accept the plan like any other.  Compared with the exact
 * brute-force plane of dm_list the pulse is smeared by about
 * 2*K*dDM*df_s/F_s^3 (Eq. sb_smear).
 *  n0        fine DMs per coarse DM, 1 .. 32 (n0 = 1: the brute-force plane)
 *  nsub      1 .. nchan subbands
 *  fs_mode   AF_FS_MEDIAN: F_s = median of the subband's channel centres
 *            (mean of the two middle ones for an even count);
 *            AF_FS_INVSQ: 1/F_s^2 = mean of 1/f_c^2 over the subband
 *  block_len the time block L of the paper's blocking (Eq. L1): af_dedisperse
 *            runs stage 1 and stage 2 once per L outputs, and the plan holds a
 *            stage-1 scratch of ncoarse*nsub*(L + max R) elements (uint16 when
 *            every subband has at most 257 channels, else uint32); 0 chooses the
 *            largest multiple of 4096 up to 2^18 that keeps it within 1 GiB.
 *  dm_list   non-decreasing, each >= 0 (AF_EINVAL otherwise)
 * Other arguments and errors as af_plan. */
#define AF_FS_MEDIAN 0
#define AF_FS_INVSQ  1
int af_plan_subband(af_plan_t* out, int nchan, double f_lo, double f_hi, double tsamp,
                    const double* dm_list, int ndm, int n0, int nsub, int fs_mode, int64_t block_len);

/* Tables of a subband plan (AF_EINVAL for a plain plan); every output may be
 * NULL: n0, nsub, ncoarse = ceil(ndm/n0), first int32 [nsub+1], fs double
 * [nsub] (MHz), coarse_delays int32 [ncoarse][nchan], residuals int32
 * [ndm][nsub], block_len = L in use. */
int af_plan_subband_info(af_plan_t plan, int* n0, int* nsub, int* ncoarse, int32_t* first, double* fs,
                         int32_t* coarse_delays, int32_t* residuals, int64_t* block_len);

/* ---- dedispersion: Sec. 2.3, the brute-force sum over channels ---------- *
 *     Y[d][t] = sum_{c} X[c][t + D[d][c]],   0 <= t < nout = nsamp - Dmax
 * exact in int32 (requires 255 * nchan < 2^31).
 *  d_in     uint8 [nchan][nsamp] (channel-major), base 16-byte aligned
 *  nsamp    samples per channel (row pitch of d_in), > Dmax
 *  d_plane  int32 [ndm][nout] output (row pitch nout)
 *  d_stats  optional af_rowstats_t [ndm] output (may be NULL)
 * Enqueued on `stream`.  Brute-force plans run the group-row kernels once
 * af_dedisperse_reserve (or af_search_reserve) has reserved their row buffer,
 * else the channel tile kernel; both give the same plane.  Never allocates.
 * AF_EINVAL for a NULL buffer, a d_in not 16-byte aligned, nsamp <= Dmax or
 * nout > 2^31 - 1; AF_ECUDA if the launch fails.  A device wait that ran out
 * (AF_ETIMEOUT) is reported by af_plan_check, which waits for the device. */
int af_dedisperse(af_plan_t plan, const uint8_t* d_in, int64_t nsamp,
                  int32_t* d_plane, af_rowstats_t* d_stats, void* stream);

/* Reserves the group-row buffer of a brute-force plan (af_plan_kernel path
 * AF_PATH_PAIRS) for inputs of up to max_nsamp samples, if a cost model
 * (rates measured on GB300) predicts group rows faster than the channel tile
 * kernel; of groups of 2, 3 and 4 channels it takes the fastest.  The
 * time-block length is the longest whose rows (uint16, one per group and
 * distinct tuple of relative delays, each the block length + the delay span of
 * its DMs long) fit the row budget (AFGB_PAIR_BUDGET_MB at plan creation,
 * default min(48 GiB, 1/5 of device memory)); later calls of any length run in
 * as many time blocks as they need.  Allocates and uploads synchronously (waits for the
 * device when it replaces a reservation); AF_OK without effect for plans that
 * cannot use group rows.  AF_EINVAL if max_nsamp <= Dmax, AF_ENOMEM / AF_ECUDA
 * on allocation failure.  Not a step of the paper's method: the same sum,
 * grouped. */
int af_dedisperse_reserve(af_plan_t plan, int64_t max_nsamp);
/* Device bytes af_dedisperse_reserve(plan, max_nsamp) would allocate (the
 * group-row buffer; 0 where the channel tile kernel serves the plan), without
 * allocating or changing anything.  AF_EINVAL if max_nsamp <= Dmax or bytes
 * is NULL. */
int af_dedisperse_workspace_size(af_plan_t plan, int64_t max_nsamp, size_t* bytes);

/* Stage timing of the group-row path (measurement aid, not a step of the
 * paper's method).  af_dedisperse_timing(plan, n) creates events for n call
 * slots (0 <= n <= 4096; 0 turns timing off) after waiting for the device;
 * every later af_dedisperse call on the group-row path records, in slot
 * (calls since then) mod n, events on its stream around stage 1 (row sums)
 * and stage 2 (tiles) of each of its first 8 time blocks.
 * af_dedisperse_times(plan, i, ...) waits for slot i's events and returns the
 * summed stage times in ms, the row-buffer bytes that call wrote and the
 * row-window bytes its stage 2 copied into shared memory (any output may be
 * NULL); AF_EINVAL for a slot outside 0..n-1. */
int af_dedisperse_timing(af_plan_t plan, int ncalls);
int af_dedisperse_times(af_plan_t plan, int call, float* rows_ms, float* tiles_ms, int64_t* row_bytes,
                        int64_t* copy_bytes);

/* Row sums of a plane [ndm][nout] into d_stats [ndm] (see af_rowstats_t).
 * Enqueued on `stream`.  AF_EINVAL for a NULL buffer or nout outside
 * 1..2^31-1. */
int af_rowstats(af_plan_t plan, const int32_t* d_plane, int64_t nout,
                af_rowstats_t* d_stats, void* stream);

/* ---- boxcar matched filter and S/N (step (iii), Sec. 1) ----------------- *
 * For every row d and time t, over the widths w in `widths` whose window
 * t .. t+w-1 fits in the row:
 *     B_w = sum_{k=t}^{t+w-1} Y[d][k]
 *     snr_w = (nout*B_w - w*S_d) / (nout * sigma_d * sqrt(w))
 * with S_d = row sum and sigma_d the population standard deviation of the
 * row (sigma_d = 0 gives snr 0).  Writes the largest snr_w (ties to the
 * smaller width) and its index into `widths`; where no width fits,
 * -INFINITY and AF_NO_WIDTH.
 *  d_plane     int32 [ndm][nout]
 *  d_stats     row sums from af_dedisperse/af_rowstats, or NULL: then the
 *              library computes them into the plan's scratch first
 *  widths      HOST array of nw strictly ascending widths, 1 <= w <= nout,
 *              w <= 8192, nw <= AF_MAX_WIDTHS, and w * 255 * nchan < 2^32
 *  d_best_snr  float [ndm][nout] output
 *  d_best_w    uint8 [ndm][nout] output (may be NULL)
 * Uses the plan's scratch (per-row normalisation constants); never allocates.
 * Enqueued on `stream`.  AF_EINVAL for a NULL plane or S/N buffer, nout
 * outside 1..2^31-1 or a width list outside these rules. */
int af_boxcar_snr(af_plan_t plan, const int32_t* d_plane, int64_t nout,
                  const af_rowstats_t* d_stats, const int32_t* widths, int nw,
                  float* d_best_snr, uint8_t* d_best_w, void* stream);

/* ---- robust S/N normalisation (median / MAD) ----------------------------- *
 * The robust alternative to the mean / standard deviation of af_boxcar_snr
 * (the paper lists robust RFI statistics among the steps either side of the
 * dedispersion, Sec. 2.1; the formula here is a reading).  Per row d:
 *     median = lower median of Y[d][0..nout) (element (nout-1)/2 of the sorted row)
 *     mad    = lower median of |Y[d][t] - median|          (both exact integers)
 *     snr_w  = (B_w - w*median) / (1.482602218505602 * mad * sqrt(w))   (mad = 0: snr 0)
 * with the windows, validity, ties and best-width output of af_boxcar_snr. */
typedef struct {
    int64_t median;
    int64_t mad;
} af_robust_t;

/* Median and MAD of every row of d_plane [ndm][nout] into d_robust [ndm]. */
int af_rowstats_robust(af_plan_t plan, const int32_t* d_plane, int64_t nout, af_robust_t* d_robust,
                       void* stream);

/* Robust boxcar S/N; d_robust may be NULL (then computed into the plan's
 * scratch first).  Other arguments and outputs as af_boxcar_snr. */
int af_boxcar_snr_robust(af_plan_t plan, const int32_t* d_plane, int64_t nout, const af_robust_t* d_robust,
                         const int32_t* widths, int nw, float* d_best_snr, uint8_t* d_best_w, void* stream);

/* ---- boxcar S/N without any device allocation --------------------------- *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc (for example a real-time receiver thread, where an
 * allocation would synchronise the device and stall the stream, or an
 * application whose own memory pool already holds all device memory) and so
 * cannot create a plan.  It computes exactly what af_boxcar_snr computes with
 * d_stats = NULL, for a plane of ndm rows of nout samples summed over nchan
 * 8-bit channels (nchan bounds the window sums: w * 255 * nchan < 2^32).
 * Its scratch is a static device array inside the library, sized for
 * ndm <= AF_NOALLOC_MAX_ROWS (about 2.1 MiB, held on every GPU that loads the
 * library until the process exits); larger ndm returns AF_EINVAL.
 * It allocates nothing.  The first call on each device looks up the array's
 * address (make it before any stream capture).  All calls share the array:
 * calls whose work overlaps on the GPU race and must be serialised.
 * Arguments and outputs are as for af_boxcar_snr; widths is a host array. */
int af_boxcar_snr_noalloc(const int32_t* d_plane, int ndm, int64_t nout, int nchan,
                          const int32_t* widths, int nw, float* d_best_snr,
                          uint8_t* d_best_w, void* stream);

/* ---- DM-time slice gridding for an image detector, Sec. 2.4 -------------- *
 * The plane's time axis is cut into S = ceil(nout / ns) slices of ns columns
 * (the last one shorter; the paper's n_s = ceil(T_slice / t_samp)) and each
 * slice (ndm x w) is resampled to an M x M image (the paper uses M = 512):
 *  - both dimensions shrink (ndm > M and w > M): the exact pixel-area mean,
 *    U(i,j) = W(i,j) / (ndm w), W = sum_r sum_c ovr(i,r) ovc(j,c) X[r][c],
 *    ovr(i,r) = |[i ndm, (i+1) ndm) & [r M, (r+1) M)| (ovc likewise);
 *  - otherwise Lanczos-4 (separable; source x = (i + 0.5) n / M - 0.5, taps
 *    floor(x) - 3 .. floor(x) + 4 weighted by sinc(t) sinc(t/4), normalised,
 *    border replicated), evaluated in double;
 * then normalised per slice to 8 bits:
 *    Y = floor(255 (U - u_min) / (u_max - u_min + eps) + 1/2),  eps = 1e-6
 * on the Lanczos path; on the area path exactly from the integer sums W,
 * without eps (0 for a constant slice).  The paper's pseudo-colour map
 * (a fixed 256-entry table applied to Y) is left to the caller.
 *  d_plane int32 [ndm][nout]; d_out uint8 [S][M][M]; d_work int64 [S][2]
 *  caller-owned scratch; M in 2..4096.  AF_EINVAL if ndm * ns * 2^31 >= 2^63.
 * Enqueued on `stream`. */
int af_grid(const int32_t* d_plane, int ndm, int64_t nout, int64_t ns, int M, uint8_t* d_out, int64_t* d_work,
            void* stream);

/* ---- thresholding and compaction into a candidate list (Sec. 2) -------- *
 * (d,t) is a candidate iff best_snr[d][t] >= thresh and, with w the best
 * width at (d,t), best_snr[d][t] > best_snr[d][u] for t-w <= u < t and
 * best_snr[d][t] >= best_snr[d][u] for t < u <= t+w (a local maximum along
 * time; ties go to the earliest t).  Candidates are appended to d_out in no
 * particular order; *d_count receives the TOTAL number found (it may exceed
 * cap; only cap records are written).  d_count is overwritten, not added to.
 *  d_best_snr, d_best_w  outputs of af_boxcar_snr ([ndm][nout])
 *  widths, nw            the same host width list
 *  sample0               added to t to form abs_sample
 *  d_out                 af_cand_t [cap] output; d_count int32 [1] output
 * Enqueued on `stream`.  AF_EINVAL for a NULL buffer (d_out may be NULL only
 * with cap = 0), a negative cap, nout outside 1..2^31-1, a non-finite
 * threshold or a width list af_boxcar_snr would reject. */
int af_candidates(af_plan_t plan, const float* d_best_snr, const uint8_t* d_best_w,
                  int64_t nout, const int32_t* widths, int nw, float thresh,
                  int64_t sample0, af_cand_t* d_out, int32_t cap, int32_t* d_count,
                  void* stream);

/* ---- host-side clustering (true-positive rule of Sec. 4.2) -------------- *
 * Sorts h_cands (in place) by (dm_idx, t), then keeps candidates greedily in
 * order of (snr desc, dm_idx asc, t asc), dropping any within
 * |dDM| < dm_tol AND |dTOA| < toa_tol (seconds) of one already kept.  DM
 * values come from the plan's DM list and TOA = abs_sample * tsamp.  Writes
 * the kept candidates to h_out (capacity n) in keep order and their number
 * to *n_out. */
int af_cluster(af_plan_t plan, af_cand_t* h_cands, int32_t n, double dm_tol,
               double toa_tol, af_cand_t* h_out, int32_t* n_out);

/* ---- whole search from HOST buffers ------------------------------------- *
 * Copies h_in (uint8 [nchan][nsamp], ideally pinned) to the device, runs
 * af_dedisperse -> af_boxcar_snr -> af_candidates on `stream` in the plan's
 * reserved workspace, copies the candidates back, sorts them by (dm_idx, t)
 * and returns after the stream has been synchronised.  *h_count = total
 * found; AF_EOVERFLOW (with the first cap candidates in h_out) if it exceeds
 * cap.  Requires af_search_reserve(plan, >= nsamp, >= cap) first (AF_ENOBUFS
 * otherwise); the reservation also holds a small pinned host buffer into
 * which the count, the error flag and up to 4096 candidates come back
 * together (one wait per call; longer lists take a second copy). */
int af_search_reserve(af_plan_t plan, int64_t max_nsamp, int32_t cap);
/* Device bytes af_search_reserve(plan, max_nsamp, cap) would allocate: the
 * input, plane, S/N, best-width and candidate buffers and the group-row
 * buffer; allocates nothing.  AF_EINVAL as af_search_reserve, or bytes NULL. */
int af_search_workspace_size(af_plan_t plan, int64_t max_nsamp, int32_t cap, size_t* bytes);
/* Phase timing of af_search (measurement aid, not a step of the paper's
 * method): with af_search_timing(plan, 1), every af_search call records
 * events on its stream; af_search_times returns, for the last call, the time
 * until the first time block's input was in (the wait of the copy), the
 * dedispersion from there (with the rest of the copy overlapped) and the
 * S/N + candidate kernels, in ms (outputs may be NULL).  AF_EINVAL if timing
 * was never enabled. */
int af_search_timing(af_plan_t plan, int enable);
int af_search_times(af_plan_t plan, float* wait_ms, float* dedisp_ms, float* snr_ms);
int af_search(af_plan_t plan, const uint8_t* h_in, int64_t nsamp,
              const int32_t* widths, int nw, float thresh,
              af_cand_t* h_out, int32_t cap, int32_t* h_count, void* stream);

/* ---- many beams in one persistent launch, replayed as a CUDA graph ------ *
 * The paper runs several antenna streams on one GPU (Sec. 4.3); here each
 * beam is an independent search (its own band, sampling, DM list, length,
 * widths and threshold).  All beams' dedispersion runs either as ONE
 * persistent channel-tile kernel that takes (beam, DM block, time tile) items
 * from a work counter, or beam after beam, each on its single-plan path (pair
 * rows, see af_dedisperse_reserve, sharing one row buffer where the beam's
 * plan uses them), whichever the build-time
 * autotuner measures faster; then every beam's boxcar S/N and candidate
 * compaction; all of it one CUDA graph.  Results are identical to
 * af_dedisperse / af_boxcar_snr / af_candidates on each beam alone. */
typedef struct af_batch_s* af_batch_t;

typedef struct {
    int nchan;              /* channels of this beam                          */
    double f_lo, f_hi;      /* band edges as for af_plan                      */
    double tsamp;           /* sampling interval, s                           */
    const double* dm_list;  /* host, ndm trial DMs (copied)                   */
    int ndm;
    const uint8_t* d_in;    /* DEVICE uint8 [nchan][nsamp], 16-byte aligned,
                               caller-owned; read at every af_batch_run      */
    int64_t nsamp;
    const int32_t* widths;  /* host, nw strictly ascending widths (copied)    */
    int nw;
    float thresh;           /* S/N threshold of the candidate step            */
    int32_t cap;            /* candidate capacity of this beam                */
} af_beam_desc_t;

/* Builds the batch: one plan per beam, each beam's plane / S/N / candidate
 * buffers on the current device (AF_ENOBUFS if they need more than
 * hbm_budget bytes; 0 = no budget), and picks the dedispersion strategy by
 * timing, on these beams (their inputs must be valid device memory; their
 * contents do not matter): one persistent channel-tile launch for every
 * compiled tile shape; the beams one after another on their single-plan
 * paths (group rows sharing one row buffer of at most 16 GiB); and persistent
 * group rows -- the time axis in waves, per wave the group rows of every
 * beam's block side by side in one buffer of at most 64 GiB, then one
 * persistent launch over all beams' (DM block, tile) items -- for ring depths
 * 3 and 2 and two wave lengths.  Row buffers lie outside hbm_budget and are
 * freed again when another strategy wins.  This is the multi-beam processing
 * of Sec. 4.3 on one GPU.
 * With the environment variable AFGB_AUTOTUNE_CACHE naming a file, the
 * choice is cached there as JSON keyed by GPU name and beam shapes;
 * AFGB_BATCH_STRATEGY=tile, =pairs or =persistent limits the choice to those
 * strategies. */
int af_batch_build(af_batch_t* out, const af_beam_desc_t* beams, int nbeams, size_t hbm_budget);

/* Enqueues the whole batch on `stream`: the first call captures a CUDA graph,
 * later calls replay it (the beams' input pointers are fixed at build). */
int af_batch_run(af_batch_t batch, void* stream);

/* After the run's stream has been synchronised: copies up to cap of beam's
 * candidates (sorted by dm_idx, t) to h_out and the total to *h_count;
 * AF_EOVERFLOW if the total exceeds cap or the beam's capacity; AF_ETIMEOUT
 * if a kernel's bounded wait ran out. */
int af_batch_candidates(af_batch_t batch, int beam, af_cand_t* h_out, int32_t cap, int32_t* h_count);

/* Device buffers of one beam (owned by the batch; any pointer may be NULL). */
int af_batch_buffers(af_batch_t batch, int beam, int32_t** d_plane, float** d_snr, uint8_t** d_best_w,
                     int64_t* nout);

/* The strategy chosen by the autotuner: the persistent tile kernel's DM rows
 * per block and 128-output groups per lane; nw = 15, m = 0 for beam after
 * beam; nw = ring depth, m = -(tiles per wave) for persistent group rows; its
 * measured time (ms, 0 if read from the cache). */
int af_batch_shape(af_batch_t batch, int* nw, int* m, float* tuned_ms, int* from_cache);

/* Candidate i (0, 1, ...) the autotuner timed at build: kind 0 = persistent
 * channel tiles (p1, p2 = the shape), 1 = beam after beam (p1 = 15, p2 = 0;
 * the fair baseline of a batch on group rows: the same kernels one plan at a
 * time, no graph), 2 = persistent group rows (p1 = ring depth, p2 = tiles per
 * wave); its time in ms.  AF_EINVAL past the last candidate (none when the
 * choice came from the cache).  No counterpart in the paper. */
int af_batch_tuning(af_batch_t batch, int i, int* kind, int* p1, int* p2, float* ms);

int af_batch_destroy(af_batch_t batch);

/* ---- streaming search with continuous batching --------------------------- *
 * Every beam is a continuous stream, searched in windows of `window` samples
 * that start every hop = window - Dmax samples: consecutive windows overlap
 * by the largest delay, so their outputs (hop samples each) tile the stream
 * exactly (the paper's time blocking with a halo of the maximum shift, Eq. L1
 * of Sec. 2.3, applied across chunks).  The overlap of each beam stays on the
 * device.  Requests are admitted into slots whose number the HBM budget sets;
 * a dispatcher thread runs every admitted window together (their
 * dedispersion -- window after window on group rows, see
 * af_dedisperse_reserve, when the plan uses them and the budget holds the
 * row buffer next to one slot; else one persistent channel-tile launch --
 * then each window's S/N and candidates), so requests that arrive while
 * others run join the next dispatch. */
typedef struct af_stream_s* af_stream_t;

typedef struct {
    int nbeams;             /* independent streams                              */
    int nchan;              /* all beams share band, sampling and DM list       */
    double f_lo, f_hi, tsamp;
    const double* dm_list;  /* host, copied */
    int ndm;
    int64_t window;         /* samples per searched window (> Dmax)             */
    const int32_t* widths;  /* host, copied */
    int nw;
    float thresh;
    int32_t cap;            /* candidates kept per window                       */
    size_t hbm_budget;      /* bytes for slots + beam state (+ the group-row buffer
                               when used); 0 = no limit                          */
    int max_slots;          /* upper bound on slots (0 = 4)                     */
    int timeout_ms;         /* af_stream_push: longest wait for a free slot;
                               0 = return AF_EAGAIN at once                     */
} af_stream_cfg_t;

typedef struct {
    int beam;
    int64_t seq;            /* chunk number of the beam (0, 1, 2, ...)          */
    int64_t sample0;        /* stream sample of output t = 0 (= seq * hop)      */
    int32_t slot;           /* pass to af_stream_release                        */
    int32_t count;          /* candidates in `cands` (<= cap)                   */
    int32_t total;          /* candidates found                                  */
    const af_cand_t* cands; /* host, sorted by (dm_idx, t); valid until release */
    double latency_ms;      /* push call -> candidates in host memory           */
    int status;             /* AF_OK, AF_EOVERFLOW (total > cap), AF_ETIMEOUT   */
} af_stream_result_t;

typedef struct {
    int64_t windows;        /* windows completed and polled                     */
    int64_t launches;       /* dispatches (one dedispersion pass over the ready windows each) */
    int max_inflight;       /* most windows admitted at once                    */
    int slots;
    double p50_ms, p99_ms, max_ms;  /* chunk-to-candidate latency               */
    double wall_s;          /* first push to last completion                    */
    double work;            /* ndm * nchan * hop per window, summed             */
    double rate;            /* work / wall_s                                    */
} af_stream_stats_t;

/* Opens the engine on the current device and starts its dispatcher thread.
 * AF_ENOBUFS if the budget cannot hold one slot plus every beam's overlap. */
int af_stream_open(af_stream_t* out, const af_stream_cfg_t* cfg);

/* Submits the next chunk of a beam: h_data is host uint8 [nchan] rows of
 * nsamp samples, `pitch` bytes apart (0 = nsamp; pinned memory copies
 * fastest), nsamp = window for the beam's first chunk
 * (seq 0) and hop afterwards, seq = the beam's next chunk number (AF_EINVAL
 * for a dropped, repeated or mis-sized chunk).  Waits up to timeout_ms for a
 * free slot (AF_EAGAIN / AF_ETIMEOUT).  Returns once the data is on the
 * device; the search itself runs asynchronously. */
int af_stream_push(af_stream_t s, int beam, const uint8_t* h_data, int64_t nsamp, int64_t pitch,
                   int64_t seq);

/* Takes the next completed window (AF_EAGAIN if none within timeout_ms).
 * The slot stays held, with its candidates and device buffers valid, until
 * af_stream_release. */
int af_stream_poll(af_stream_t s, af_stream_result_t* out, int timeout_ms);
int af_stream_release(af_stream_t s, int32_t slot);

/* Inline classification of a held window: cut-outs of the n host candidates
 * (n <= the engine's cap; typically the cluster representatives of the
 * window's candidates) from the window's device input and plane, and the
 * classifier's P(pulse) for each into h_prob[n].  Synchronous.  Calls on the
 * same engine must not overlap. */
int af_stream_classify(af_stream_t s, int32_t slot, af_model_t model, const af_cand_t* h_cands, int32_t n,
                       float* h_prob);
/* The true-positive clustering of Sec. 4.2 (as af_cluster) with the engine's DM list and sampling. */
int af_stream_cluster(af_stream_t s, af_cand_t* h_cands, int32_t n, af_cand_t* h_out, int32_t* n_out);

/* Device plane [ndm][hop] and best S/N of a held slot. */
int af_stream_result_plane(af_stream_t s, int32_t slot, int32_t** d_plane, float** d_snr, int64_t* nout);

int af_stream_info(af_stream_t s, int64_t* hop, int64_t* dmax, int* nslots);
int af_stream_stats(af_stream_t s, af_stream_stats_t* st);

/* Per-beam state for checkpoint / resume: the overlap (uint8 [nchan][Dmax]),
 * the next chunk number and the next window's first stream sample.  A beam
 * restored into a fresh engine continues exactly as if it had never stopped. */
int af_stream_snapshot(af_stream_t s, int beam, uint8_t* h_overlap, int64_t* next_seq, int64_t* next_sample);
int af_stream_restore(af_stream_t s, int beam, const uint8_t* h_overlap, int64_t next_seq, int64_t next_sample);

/* Waits for all work, stops the dispatcher and frees everything. */
int af_stream_close(af_stream_t s);

/* ---- diagnostic: measured integer issue rates ---------------------------- *
 * Not a step of the paper's method: the denominator of the dedispersion
 * roofline, measured on the current device.  Runs two short probe kernels
 * (one block of 1024 threads per SM, a few milliseconds, synchronous) and
 * returns, in thread-operations per second,
 *   add_per_s           32-bit 2-input additions (8 independent chains per thread)
 *   pattern_adds_per_s  sample additions of the dedispersion inner step: two
 *                       32-bit shared loads (4 uint8 samples each), widening
 *                       into 16-bit lanes (and-mask, byte permute) and the
 *                       paired adds, i.e. 8 sample additions per step.
 * Allocates nothing (a static device array receives the probes' results). */
int af_diag_int_rates(double* add_per_s, double* pattern_adds_per_s);
/* Shared-memory load bandwidth of the current device in bytes per second, the
 * denominator of the group-row tile kernel's roofline: one block of 1024
 * threads per SM, 8 independent lane-consecutive (bank-conflict-free) 32-bit
 * shared loads per thread and step, each added into an accumulator.  A few
 * milliseconds, synchronous; allocates nothing.  AF_EINVAL if bytes_per_s is
 * NULL. */
int af_diag_smem_rate(double* bytes_per_s);
/* Failure path of the bounded device waits, made to happen.  The ring kernels
 * (tile, group-row and subband stage-2 kernels) wait on mbarriers with at most
 * 2^18 polls; a wait that runs out raises the plan's (batch's, engine's) error
 * flag and the kernel returns, so a lost arrival surfaces as AF_ETIMEOUT and
 * never as a hang.  This probe runs the same bounded poll loop in one block of
 * 128 threads on the legacy default stream: arrive = 0 waits on a barrier that
 * nothing arrives at, so every wait gives up after `polls` polls and the call
 * returns AF_ETIMEOUT; arrive != 0 lets one thread arrive first and returns
 * AF_OK.  *ms (nullable) receives the kernel's duration, i.e. how long `polls`
 * polls of a wait that never completes take on this device.  Synchronous;
 * allocates nothing; AF_EINVAL unless 1 <= polls <= 2^24.  Not a step of the
 * paper's method. */
int af_diag_bounded_wait(int arrive, int64_t polls, float* ms);

/* ---- candidate classifier ----------------------------------------------- *
 * The paper detects pulses with a YOLOv11n network on DM-time images
 * (Sec. 2.5); its weights and data sets are not available, so the library
 * carries a small CNN instead, trained on the GPU by the library's own kernels
 * (BF16 tensor-core GEMMs, FP32 accumulation):
 * input NHWC bf16 [n][64][64][2] (channel 0 DM-time, 1 frequency-time cut-out),
 * three blocks conv3x3 (+bias) -> ReLU -> 2x2 max pool (2 -> 16 -> 32 -> 64
 * channels), global average pool, fully connected 64 -> 2, softmax; label /
 * class 1 = pulse.  bf16 values travel as uint16_t.  Parameters are fp32, flat:
 * w0 [16][3][3][2], b0 [16], w1 [32][3][3][16], b1 [32], w2 [64][3][3][32],
 * b2 [64], fw [2][64], fb [2] (23570 values). */
/* Two 64 x 64 cut-outs per candidate (adapting the gridding and min-max
 * normalisation of Sec. 2.4): time bins of b = max(1, width/2) samples, bin j
 * covering [t - 32b + jb, t - 32b + (j+1)b) (samples outside [0, nout) count 0);
 * DM-time [i][j] = bin sum of plane row dm_idx - 32 + i (zero outside the
 * plane); frequency-time [g][j] = bin sum over channel group g (nchan/64
 * channels) of X[c][s + D[dm_idx][c]]; each normalised as
 * float(v - min) / (float(max - min) + 1e-6f) and rounded to bf16.
 *  d_in [nchan][nsamp] uint8, d_plane [ndm][nout] int32 (nout = nsamp - Dmax),
 *  d_cands [n] device, d_out bf16 [n][64][64][2].  nchan must be a multiple of 64. */
int af_cutouts(af_plan_t plan, const uint8_t* d_in, int64_t nsamp, const int32_t* d_plane, int64_t nout,
               const af_cand_t* d_cands, int32_t n, uint16_t* d_out, void* stream);

/* The classifier's tensor-core GEMM (tcgen05.mma, bf16 operands, fp32
 * accumulation in tensor memory), for tests and tools; no counterpart in the
 * paper.  C[m][n] (op)= sum_k A(m,k) B(k,n)  with
 *  layout 0: A [M][K], B given as [N][K];   1: A [M][K], B [K][N];
 *         2: A given as [K][M], B [K][N];   3: A given as [K][M], B as [N][K]
 *  epi    0: C = acc;  1: C = max(acc + bias[n], 0);  2: C += acc (atomic, fp32)
 * lda / ldb = row pitch of the stored arrays in elements (multiples of 8),
 * ldc of C (fp32 [M][ldc]); K a multiple of 8; operands 16-byte aligned;
 * splits > 1 splits K across blocks (epi 2 only).  Unlike the other calls it
 * allocates a 4-byte flag and waits for the stream: AF_ETIMEOUT if one of the
 * kernel's bounded waits for its tensor-core operations ran out. */
int af_nn_gemm(int layout, int epi, const uint16_t* d_a, int lda, const uint16_t* d_b, int ldb, int M, int N, int K,
               int splits, float* d_c, int ldc, const float* d_bias, void* stream);

/* Allocates parameters, Adam state and the workspace of batches up to
 * max_batch on the current device; He-normal initial weights from `seed`. */
int af_model_create(af_model_t* out, int max_batch, uint64_t seed);
int af_model_destroy(af_model_t model);
int af_model_nparams(af_model_t model, int64_t* n);
/* Host fp32 parameter / gradient vectors in the flat order above (synchronous).
 * The classifier's convolutions run on the tcgen05 tensor cores with bounded
 * waits for their MMAs; a wait that ran out in an earlier forward / backward /
 * training call is reported here (and by af_model_save) as AF_ETIMEOUT. */
int af_model_set_params(af_model_t model, const float* h_params, int64_t n);
int af_model_get_params(af_model_t model, float* h_params, int64_t n);
int af_model_get_grads(af_model_t model, float* h_grads, int64_t n);
/* Checkpoint: JSON header line + raw little-endian fp32 parameters and Adam moments. */
int af_model_save(af_model_t model, const char* path);
int af_model_load(af_model_t model, const char* path);

/* Forward pass: d_x bf16 [n][64][64][2] (n <= max_batch, 16-byte aligned);
 * d_logits fp32 [n][2] and d_prob fp32 [n] = P(pulse) (either may be NULL). */
int af_model_forward(af_model_t model, const uint16_t* d_x, int32_t n, float* d_logits, float* d_prob,
                     void* stream);
/* Forward + backward of the mean softmax cross-entropy for labels d_y int32 [n]
 * (0/1); gradients stay in the model (af_model_get_grads); d_loss fp32 [1]. */
int af_model_backward(af_model_t model, const uint16_t* d_x, const int32_t* d_y, int32_t n, float* d_loss,
                      void* stream);
/* af_model_backward followed by one Adam step (beta1 0.9, beta2 0.999, eps 1e-8). */
int af_train_step(af_model_t model, const uint16_t* d_x, const int32_t* d_y, int32_t n, float lr, float* d_loss,
                  void* stream);
/* Cut-outs of n candidates (any n; processed max_batch at a time) and the
 * network's P(pulse) for each, into d_prob fp32 [n]. */
int af_classify(af_model_t model, af_plan_t plan, const uint8_t* d_in, int64_t nsamp, const int32_t* d_plane,
                int64_t nout, const af_cand_t* d_cands, int32_t n, float* d_prob, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* AFGB_H */
