// plan.cpp -- host side of the afgb C ABI: errors, the delay-table plan
// (Eq. coarse_delay, Sec. 2.3), argument checking, candidate clustering
// (Sec. 4.2) and the host-buffer search.
//
// Compiled with -ffp-contract=off so that the delay arithmetic is the plain
// IEEE double sequence stated in afgb.h on every host (x86_64 and aarch64).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

static thread_local std::string g_last_error;

int af_set_error(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int af_cuda_check(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return AF_OK;
    return af_set_error(e == cudaErrorMemoryAllocation ? AF_ENOMEM : AF_ECUDA, "%s: %s (%s)", what,
                        cudaGetErrorString(e), cudaGetErrorName(e));
}

int af_host_exception(const char* who)
{
    try {
        try {
            throw;
        } catch (const std::bad_alloc&) {
            return af_set_error(AF_ENOMEM, "%s: host allocation failed", who);
        } catch (const std::exception& e) {
            return af_set_error(AF_EINVAL, "%s: %s", who, e.what());
        } catch (...) {
            return af_set_error(AF_EINVAL, "%s: unexpected host exception", who);
        }
    } catch (...) {
        return AF_ENOMEM;  // recording the message failed as well
    }
}

extern "C" const char* af_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* af_version(void) { return "afgb 0.1 (sm_103a)"; }

int af_check_plan(af_plan_t p)
{
    if (!p) return af_set_error(AF_EINVAL, "null plan");
    return AF_OK;
}

// Dispersion constant, Eq. (KDM): seconds when frequencies are in MHz.
static const double kKDM = 4.148808e3;

// Candidates af_search copies back together with their count.
static const int32_t kSearchStage = 4096;
// af_search copies its input in channel bands: a band needs, for the outputs
// before T, the columns before T + (its largest delay), so the low-delay bands
// of the first time block arrive sooner than a copy of every channel up to
// T + Dmax would (half the bytes on a 1000-1500 MHz band).
static const int kSearchBands = 8;

static void search_bands(af_plan_t p)
{
    const int nb = std::min(kSearchBands, p->nchan);
    p->ws_band.assign(nb + 1, 0);
    p->ws_band_dmax.assign(nb, 0);
    for (int j = 0; j <= nb; j++) p->ws_band[j] = (int32_t)((int64_t)p->nchan * j / nb);
    for (int j = 0; j < nb; j++) {
        int32_t m = 0;
        for (int d = 0; d < p->ndm; d++)
            for (int c = p->ws_band[j]; c < p->ws_band[j + 1]; c++)
                m = std::max(m, p->delays[(size_t)d * p->nchan + c]);
        p->ws_band_dmax[j] = m;
    }
}

// Copies, band by band on the copy stream, every input column that the
// outputs before `end` read (all of them when `last`); col[j] = the columns
// band j already has.
static int search_copy_upto(af_plan_t p, const uint8_t* h_in, int64_t nsamp, int64_t end, bool last, int64_t* col)
{
    const int nb = (int)p->ws_band_dmax.size();
    for (int j = 0; j < nb; j++) {
        const int64_t need = last ? nsamp : std::min<int64_t>(nsamp, end + p->ws_band_dmax[j]);
        if (need <= col[j]) continue;
        const size_t c0 = (size_t)p->ws_band[j], nc = (size_t)(p->ws_band[j + 1] - p->ws_band[j]);
        AF_CUDA(cudaMemcpy2DAsync(p->ws_in + c0 * nsamp + col[j], (size_t)nsamp, h_in + c0 * nsamp + col[j],
                                  (size_t)nsamp, (size_t)(need - col[j]), nc, cudaMemcpyHostToDevice, p->ws_copy));
        col[j] = need;
    }
    return AF_OK;
}

static void free_search_ws(af_plan_t p)
{
    cudaFree(p->ws_in);
    cudaFree(p->ws_plane);
    cudaFree(p->ws_snr);
    cudaFree(p->ws_bw);
    cudaFree(p->ws_cands);
    cudaFree(p->ws_count);
    cudaFreeHost(p->ws_host);
    if (p->ws_copy) cudaStreamDestroy(p->ws_copy);
    for (cudaEvent_t& e : p->ws_ev)
        if (e) cudaEventDestroy(e), e = nullptr;
    for (cudaEvent_t& e : p->ws_tev)
        if (e) cudaEventDestroy(e), e = nullptr;
    p->ws_timing = false;
    p->ws_copy = nullptr;
    p->ws_in = nullptr;
    p->ws_plane = nullptr;
    p->ws_snr = nullptr;
    p->ws_bw = nullptr;
    p->ws_cands = nullptr;
    p->ws_count = nullptr;
    p->ws_host = nullptr;
    p->ws_stage = 0;
    p->ws_nsamp = 0;
    p->ws_cap = 0;
}

static void free_plan(af_plan_t p)
{
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    cudaFree(p->d_delays);
    af_tile_tables_free(&p->tile);
    af_pairs_free(&p->pairs);
    af_pairs_free(&p->alt[0]);
    af_pairs_free(&p->alt[1]);
    af_sb_free(p);
    cudaFree(p->d_err);
    cudaFree(p->d_stats);
    cudaFree(p->d_rowconst);
    free_search_ws(p);
    if (cur != p->device) cudaSetDevice(cur);
    delete p;
}

static int check_plan_args(const char* who, int nchan, double f_lo, double f_hi, double tsamp,
                           const double* dm_list, int ndm)
{
    if (nchan < 1 || nchan > 65536) return af_set_error(AF_EINVAL, "%s: nchan %d out of range", who, nchan);
    if (ndm < 1 || ndm > (1 << 20)) return af_set_error(AF_EINVAL, "%s: ndm %d out of range", who, ndm);
    if (!dm_list) return af_set_error(AF_EINVAL, "%s: dm_list is NULL", who);
    if (!(f_lo > 0.0) || !(f_hi > 0.0) || f_lo == f_hi || !isfinite(f_lo) || !isfinite(f_hi))
        return af_set_error(AF_EINVAL, "%s: bad band edges %g %g", who, f_lo, f_hi);
    if (!(tsamp > 0.0) || !isfinite(tsamp)) return af_set_error(AF_EINVAL, "%s: bad tsamp %g", who, tsamp);
    for (int d = 0; d < ndm; d++)
        if (!(dm_list[d] >= 0.0) || !isfinite(dm_list[d]))
            return af_set_error(AF_EINVAL, "%s: dm_list[%d] = %g is not a finite value >= 0", who, d, dm_list[d]);
    return AF_OK;
}

// Channel-centre frequency and reference frequency (top band edge).
static double chan_freq(int c, int nchan, double f_lo, double f_hi)
{
    const double df = (f_hi - f_lo) / (double)nchan;
    return f_lo + ((double)c + 0.5) * df;
}

// Eq. (coarse_delay) for a list of DMs: D = round(K*DM/tsamp * (1/fc^2 - 1/fref^2)),
// channel centres, f_ref = top band edge, round half away from zero.
// The table covers channels [c0, c0 + nchan) of a band of ntot channels.
static int delay_rows(const char* who, int nchan, double f_lo, double f_hi, double tsamp, const double* dms,
                      int n, int32_t* out, int32_t* dmax, int c0 = 0, int ntot = 0)
{
    if (ntot == 0) ntot = nchan;
    const double fr = f_lo > f_hi ? f_lo : f_hi;
    std::vector<double> bterm(nchan);
    for (int c = 0; c < nchan; c++) {
        const double fc = chan_freq(c0 + c, ntot, f_lo, f_hi);
        bterm[c] = 1.0 / (fc * fc) - 1.0 / (fr * fr);
    }
    int32_t mx = 0;
    for (int d = 0; d < n; d++) {
        const double a = (kKDM * dms[d]) / tsamp;
        for (int c = 0; c < nchan; c++) {
            const double x = a * bterm[c];
            if (!(x < 2147483647.0))
                return af_set_error(AF_EINVAL, "%s: delay of dm %g channel %d exceeds int32", who, dms[d], c);
            const int32_t D = (int32_t)llround(x);
            out[(size_t)d * nchan + c] = D;
            mx = D > mx ? D : mx;
        }
    }
    if (dmax) *dmax = mx;
    return AF_OK;
}

static af_plan_s* new_plan(int nchan, double f_lo, double f_hi, double tsamp, const double* dm_list, int ndm)
{
    af_plan_s* p = new (std::nothrow) af_plan_s();
    if (!p) return nullptr;
    p->nchan = nchan;
    p->ndm = ndm;
    p->f_lo = f_lo;
    p->f_hi = f_hi;
    p->tsamp = tsamp;
    try {
        p->dms.assign(dm_list, dm_list + ndm);
        p->delays.resize((size_t)ndm * nchan);
    } catch (...) {
        delete p;
        return nullptr;
    }
    return p;
}

// Device side common to every plan: table upload, scratch, tile tables.
// Frees the plan on failure.
static int plan_finish(af_plan_s* p, const char* who)
{
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return af_cuda_check(e, who);
    }
    cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (const char* k = getenv("AFGB_DEDISP_KERNEL")) {
        p->force_simple = strcmp(k, "simple") == 0;
        p->force_brute = strcmp(k, "brute") == 0;
        p->force_tile = strcmp(k, "tile") == 0;
        p->force_pairs = strcmp(k, "pairs") == 0;
    }
    if (const char* g = getenv("AFGB_PAIR_GROUP")) {
        const int v = atoi(g);
        p->force_group = v >= 2 && v <= 4 ? v : 0;
    }
    const size_t tbytes = (size_t)p->ndm * p->nchan * sizeof(int32_t);
    int rc = AF_OK;
    if ((e = cudaMalloc(&p->d_delays, tbytes)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_delays, p->delays.data(), tbytes, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_stats, (size_t)p->ndm * sizeof(af_rowstats_t))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_rowconst, (size_t)p->ndm * AF_MAX_WIDTHS * sizeof(af_rowconst_t))) != cudaSuccess) {
        rc = af_cuda_check(e, "plan: device allocation/upload");
    }
    if (rc == AF_OK) rc = af_prepare_dedisp_tables(p);
    if (rc == AF_OK && p->sb_nsub > 0) rc = af_sb_prepare(p);
    if (rc != AF_OK) free_plan(p);
    return rc;
}

extern "C" int af_plan(af_plan_t* out, int nchan, double f_lo, double f_hi, double tsamp,
                       const double* dm_list, int ndm)
try {
    if (!out) return af_set_error(AF_EINVAL, "af_plan: out is NULL");
    *out = nullptr;
    if (int rc = check_plan_args("af_plan", nchan, f_lo, f_hi, tsamp, dm_list, ndm)) return rc;
    af_plan_s* p = new_plan(nchan, f_lo, f_hi, tsamp, dm_list, ndm);
    if (!p) return af_set_error(AF_ENOMEM, "af_plan: host allocation failed");
    if (int rc = delay_rows("af_plan", nchan, f_lo, f_hi, tsamp, dm_list, ndm, p->delays.data(), &p->dmax)) {
        delete p;
        return rc;
    }
    if (int rc = plan_finish(p, "af_plan")) return rc;
    *out = p;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_plan");
}

extern "C" int af_plan_channels(af_plan_t* out, int nchan, double f_lo, double f_hi, double tsamp,
                                const double* dm_list, int ndm, int c0, int c1)
try {
    static const char* who = "af_plan_channels";
    if (!out) return af_set_error(AF_EINVAL, "%s: out is NULL", who);
    *out = nullptr;
    if (int rc = check_plan_args(who, nchan, f_lo, f_hi, tsamp, dm_list, ndm)) return rc;
    if (c0 < 0 || c1 > nchan || c1 <= c0)
        return af_set_error(AF_EINVAL, "%s: channel range [%d, %d) not inside [0, %d)", who, c0, c1, nchan);
    const int n = c1 - c0;
    af_plan_s* p = new_plan(n, f_lo, f_hi, tsamp, dm_list, ndm);
    if (!p) return af_set_error(AF_ENOMEM, "%s: host allocation failed", who);
    if (int rc = delay_rows(who, n, f_lo, f_hi, tsamp, dm_list, ndm, p->delays.data(), &p->dmax, c0, nchan)) {
        delete p;
        return rc;
    }
    if (int rc = plan_finish(p, who)) return rc;
    *out = p;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_plan_channels");
}

// Representative frequency of channels [c0, c1), Sec. 2.3: the median of the
// channel centres (mean of the two middle ones for an even count), or the
// frequency whose 1/F^2 is the mean of 1/f_c^2.
static double subband_freq(int nchan, double f_lo, double f_hi, int c0, int c1, int mode)
{
    const int n = c1 - c0;
    if (mode == AF_FS_MEDIAN) {
        std::vector<double> f(n);
        for (int i = 0; i < n; i++) f[i] = chan_freq(c0 + i, nchan, f_lo, f_hi);
        std::sort(f.begin(), f.end());
        return (n % 2) ? f[n / 2] : 0.5 * (f[n / 2 - 1] + f[n / 2]);
    }
    double acc = 0.0;
    for (int c = c0; c < c1; c++) {
        const double fc = chan_freq(c, nchan, f_lo, f_hi);
        acc += 1.0 / (fc * fc);
    }
    return 1.0 / sqrt(acc / (double)n);
}

extern "C" int af_plan_subband(af_plan_t* out, int nchan, double f_lo, double f_hi, double tsamp,
                               const double* dm_list, int ndm, int n0, int nsub, int fs_mode, int64_t block_len)
try {
    static const char* who = "af_plan_subband";
    if (!out) return af_set_error(AF_EINVAL, "%s: out is NULL", who);
    *out = nullptr;
    if (int rc = check_plan_args(who, nchan, f_lo, f_hi, tsamp, dm_list, ndm)) return rc;
    if (n0 < 1 || n0 > 32) return af_set_error(AF_EINVAL, "%s: n0 %d not in 1..32", who, n0);
    if (nsub < 1 || nsub > nchan) return af_set_error(AF_EINVAL, "%s: nsub %d not in 1..nchan", who, nsub);
    if (fs_mode != AF_FS_MEDIAN && fs_mode != AF_FS_INVSQ)
        return af_set_error(AF_EINVAL, "%s: unknown fs_mode %d", who, fs_mode);
    if (block_len < 0 || block_len > ((int64_t)1 << 30))
        return af_set_error(AF_EINVAL, "%s: block_len %lld out of range", who, (long long)block_len);
    for (int m = 1; m < ndm; m++)
        if (!(dm_list[m] >= dm_list[m - 1]))
            return af_set_error(AF_EINVAL, "%s: dm_list must be non-decreasing (entry %d)", who, m);
    af_plan_s* p = new_plan(nchan, f_lo, f_hi, tsamp, dm_list, ndm);
    if (!p) return af_set_error(AF_ENOMEM, "%s: host allocation failed", who);
    p->sb_n0 = n0;
    p->sb_nsub = nsub;
    p->sb_mode = fs_mode;
    p->sb_ncoarse = (ndm + n0 - 1) / n0;
    try {
        // partition: subband s = channels [floor(s*nchan/nsub), floor((s+1)*nchan/nsub))
        p->sb_first.resize(nsub + 1);
        for (int s = 0; s <= nsub; s++) p->sb_first[s] = (int32_t)(((int64_t)s * nchan) / nsub);
        p->sb_F.resize(nsub);
        for (int s = 0; s < nsub; s++)
            p->sb_F[s] = subband_freq(nchan, f_lo, f_hi, p->sb_first[s], p->sb_first[s + 1], fs_mode);
        // coarse DMs dm_list[j*n0] and their delays, Eq. (coarse_delay)
        p->sb_cdms.resize(p->sb_ncoarse);
        for (int j = 0; j < p->sb_ncoarse; j++) p->sb_cdms[j] = dm_list[j * n0];
        p->sb_dc.resize((size_t)p->sb_ncoarse * nchan);
        p->sb_r.resize((size_t)ndm * nsub);
    } catch (...) {
        delete p;
        return af_set_error(AF_ENOMEM, "%s: host allocation failed", who);
    }
    if (int rc = delay_rows(who, nchan, f_lo, f_hi, tsamp, p->sb_cdms.data(), p->sb_ncoarse, p->sb_dc.data(),
                            nullptr)) {
        delete p;
        return rc;
    }
    // residual shifts, Eq. (residual): R = round(K*dDM/tsamp * (1/F_s^2 - 1/fref^2))
    const double fr = f_lo > f_hi ? f_lo : f_hi;
    int32_t rmax = 0;
    for (int s = 0; s < nsub; s++) {
        const double F = p->sb_F[s];
        const double b = 1.0 / (F * F) - 1.0 / (fr * fr);
        for (int m = 0; m < ndm; m++) {
            const double ddm = dm_list[m] - dm_list[(m / n0) * n0];
            const double a = (kKDM * ddm) / tsamp;
            const double x = a * b;
            if (!(x < 2147483647.0)) {
                delete p;
                return af_set_error(AF_EINVAL, "%s: residual shift of dm %g exceeds int32", who, dm_list[m]);
            }
            const int32_t r = (int32_t)llround(x);
            p->sb_r[(size_t)m * nsub + s] = r;
            rmax = r > rmax ? r : rmax;
        }
    }
    p->sb_rmax = rmax;
    // effective delay table Deff[m][c] = D[j(m)][c] + R[m][s(c)]
    int32_t dmax = 0;
    for (int s = 0; s < nsub; s++)
        for (int c = p->sb_first[s]; c < p->sb_first[s + 1]; c++)
            for (int m = 0; m < ndm; m++) {
                const int64_t v = (int64_t)p->sb_dc[(size_t)(m / n0) * nchan + c] + p->sb_r[(size_t)m * nsub + s];
                if (v > INT32_MAX) {
                    delete p;
                    return af_set_error(AF_EINVAL, "%s: effective delay exceeds int32", who);
                }
                p->delays[(size_t)m * nchan + c] = (int32_t)v;
                dmax = (int32_t)v > dmax ? (int32_t)v : dmax;
            }
    p->dmax = dmax;
    p->sb_L = block_len;
    if (int rc = plan_finish(p, who)) return rc;
    *out = p;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_plan_subband");
}

extern "C" int af_plan_subband_info(af_plan_t p, int* n0, int* nsub, int* ncoarse, int32_t* first, double* fs,
                                    int32_t* coarse_delays, int32_t* residuals, int64_t* block_len)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (p->sb_nsub == 0) return af_set_error(AF_EINVAL, "af_plan_subband_info: not a subband plan");
    if (n0) *n0 = p->sb_n0;
    if (nsub) *nsub = p->sb_nsub;
    if (ncoarse) *ncoarse = p->sb_ncoarse;
    if (first) memcpy(first, p->sb_first.data(), p->sb_first.size() * sizeof(int32_t));
    if (fs) memcpy(fs, p->sb_F.data(), p->sb_F.size() * sizeof(double));
    if (coarse_delays) memcpy(coarse_delays, p->sb_dc.data(), p->sb_dc.size() * sizeof(int32_t));
    if (residuals) memcpy(residuals, p->sb_r.data(), p->sb_r.size() * sizeof(int32_t));
    if (block_len) *block_len = p->sb_L;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_plan_subband_info");
}

extern "C" int af_plan_destroy(af_plan_t plan)
try {
    free_plan(plan);
    return AF_OK;
} catch (...) {
    return af_host_exception("af_plan_destroy");
}

extern "C" int af_plan_delays(af_plan_t p, int32_t* host_out, int32_t* dmax)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (host_out) memcpy(host_out, p->delays.data(), p->delays.size() * sizeof(int32_t));
    if (dmax) *dmax = p->dmax;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_plan_delays");
}

extern "C" int af_plan_info(af_plan_t p, int* nchan, int* ndm, int32_t* dmax, double* tsamp)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (nchan) *nchan = p->nchan;
    if (ndm) *ndm = p->ndm;
    if (dmax) *dmax = p->dmax;
    if (tsamp) *tsamp = p->tsamp;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_plan_info");
}

extern "C" int af_plan_check(af_plan_t p)
try {
    if (int rc = af_check_plan(p)) return rc;
    int flag = 0;
    AF_CUDA(cudaDeviceSynchronize());
    AF_CUDA(cudaMemcpy(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        AF_CUDA(cudaMemset(p->d_err, 0, sizeof(int)));
        return af_set_error(AF_ETIMEOUT, "a kernel's bounded wait for an asynchronous copy ran out");
    }
    return AF_OK;
} catch (...) {
    return af_host_exception("af_plan_check");
}

extern "C" int af_plan_nout(af_plan_t p, int64_t nsamp, int64_t* nout)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (!nout) return af_set_error(AF_EINVAL, "af_plan_nout: nout is NULL");
    int64_t n = nsamp - (int64_t)p->dmax;
    if (n <= 0)
        return af_set_error(AF_EINVAL, "af_plan_nout: nsamp %lld <= Dmax %d", (long long)nsamp, p->dmax);
    *nout = n;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_plan_nout");
}

int af_check_widths(af_plan_t p, const int32_t* widths, int nw, int64_t nout, af_widths_t* out)
{
    return af_check_widths_nchan(p->nchan, widths, nw, nout, out);
}

int af_check_widths_nchan(int nchan, const int32_t* widths, int nw, int64_t nout, af_widths_t* out)
{
    if (!widths) return af_set_error(AF_EINVAL, "widths is NULL");
    if (nw < 1 || nw > AF_MAX_WIDTHS) return af_set_error(AF_EINVAL, "nw %d not in 1..%d", nw, AF_MAX_WIDTHS);
    memset(out, 0, sizeof *out);
    for (int i = 0; i < nw; i++) {
        if (widths[i] < 1 || (i > 0 && widths[i] <= widths[i - 1]))
            return af_set_error(AF_EINVAL, "widths must be strictly ascending and >= 1");
        if ((int64_t)widths[i] > nout)
            return af_set_error(AF_EINVAL, "width %d exceeds nout %lld", widths[i], (long long)nout);
        if ((double)widths[i] * 255.0 * (double)nchan >= 4294967296.0)
            return af_set_error(AF_EINVAL, "width %d too large for exact 32-bit window sums", widths[i]);
        if (widths[i] > 8192) return af_set_error(AF_EINVAL, "width %d > 8192 not supported", widths[i]);
        out->w[i] = widths[i];
    }
    out->n = nw;
    out->small = (double)widths[nw - 1] * 255.0 * (double)nchan < 2147483648.0 ? 1 : 0;
    return AF_OK;
}

static int check_nout(af_plan_t p, int64_t nsamp, int64_t* nout)
{
    int64_t n = nsamp - (int64_t)p->dmax;
    if (n <= 0)
        return af_set_error(AF_EINVAL, "nsamp %lld must exceed Dmax %d", (long long)nsamp, p->dmax);
    if (n > INT32_MAX) return af_set_error(AF_EINVAL, "nout %lld too large", (long long)n);
    *nout = n;
    return AF_OK;
}

extern "C" int af_dedisperse(af_plan_t p, const uint8_t* d_in, int64_t nsamp, int32_t* d_plane,
                             af_rowstats_t* d_stats, void* stream)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (!d_in || !d_plane) return af_set_error(AF_EINVAL, "af_dedisperse: NULL buffer");
    if (((uintptr_t)d_in & 15) != 0) return af_set_error(AF_EINVAL, "af_dedisperse: d_in not 16-byte aligned");
    if (255.0 * p->nchan >= 2147483648.0) return af_set_error(AF_EINVAL, "af_dedisperse: too many channels");
    int64_t nout = 0;
    if (int rc = check_nout(p, nsamp, &nout)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    return af_launch_dedisperse(p, d_in, nsamp, nout, d_plane, d_stats, s);
} catch (...) {
    return af_host_exception("af_dedisperse");
}

extern "C" int af_rowstats(af_plan_t p, const int32_t* d_plane, int64_t nout, af_rowstats_t* d_stats,
                           void* stream)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (!d_plane || !d_stats) return af_set_error(AF_EINVAL, "af_rowstats: NULL buffer");
    if (nout < 1 || nout > INT32_MAX) return af_set_error(AF_EINVAL, "af_rowstats: bad nout");
    return af_launch_rowstats(d_plane, p->ndm, nout, d_stats, (cudaStream_t)stream);
} catch (...) {
    return af_host_exception("af_rowstats");
}

extern "C" int af_boxcar_snr(af_plan_t p, const int32_t* d_plane, int64_t nout, const af_rowstats_t* d_stats,
                             const int32_t* widths, int nw, float* d_best_snr, uint8_t* d_best_w, void* stream)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (!d_plane || !d_best_snr) return af_set_error(AF_EINVAL, "af_boxcar_snr: NULL buffer");
    if (nout < 1 || nout > INT32_MAX) return af_set_error(AF_EINVAL, "af_boxcar_snr: bad nout");
    af_widths_t w;
    if (int rc = af_check_widths(p, widths, nw, nout, &w)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (!d_stats) {
        if (int rc = af_launch_rowstats(d_plane, p->ndm, nout, p->d_stats, s)) return rc;
        d_stats = p->d_stats;
    }
    return af_launch_boxcar(d_plane, p->ndm, nout, d_stats, w, p->d_rowconst, d_best_snr, d_best_w, s);
} catch (...) {
    return af_host_exception("af_boxcar_snr");
}

extern "C" int af_rowstats_robust(af_plan_t p, const int32_t* d_plane, int64_t nout, af_robust_t* d_robust,
                                  void* stream)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (!d_plane || !d_robust) return af_set_error(AF_EINVAL, "af_rowstats_robust: NULL buffer");
    if (nout < 1 || nout > INT32_MAX) return af_set_error(AF_EINVAL, "af_rowstats_robust: bad nout");
    return af_launch_row_robust(d_plane, p->ndm, nout, d_robust, (cudaStream_t)stream);
} catch (...) {
    return af_host_exception("af_rowstats_robust");
}

extern "C" int af_boxcar_snr_robust(af_plan_t p, const int32_t* d_plane, int64_t nout, const af_robust_t* d_robust,
                                    const int32_t* widths, int nw, float* d_best_snr, uint8_t* d_best_w,
                                    void* stream)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (!d_plane || !d_best_snr) return af_set_error(AF_EINVAL, "af_boxcar_snr_robust: NULL buffer");
    if (nout < 1 || nout > INT32_MAX) return af_set_error(AF_EINVAL, "af_boxcar_snr_robust: bad nout");
    af_widths_t w;
    if (int rc = af_check_widths(p, widths, nw, nout, &w)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (!d_robust) {
        // the plan's row-sum scratch has the same size and alignment
        af_robust_t* scratch = reinterpret_cast<af_robust_t*>(p->d_stats);
        if (int rc = af_launch_row_robust(d_plane, p->ndm, nout, scratch, s)) return rc;
        d_robust = scratch;
    }
    return af_launch_boxcar_robust(d_plane, p->ndm, nout, d_robust, w, p->d_rowconst, d_best_snr, d_best_w, s);
} catch (...) {
    return af_host_exception("af_boxcar_snr_robust");
}

extern "C" int af_candidates(af_plan_t p, const float* d_best_snr, const uint8_t* d_best_w, int64_t nout,
                             const int32_t* widths, int nw, float thresh, int64_t sample0, af_cand_t* d_out,
                             int32_t cap, int32_t* d_count, void* stream)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (!d_best_snr || !d_best_w || !d_count || (cap > 0 && !d_out))
        return af_set_error(AF_EINVAL, "af_candidates: NULL buffer");
    if (cap < 0) return af_set_error(AF_EINVAL, "af_candidates: negative cap");
    if (nout < 1 || nout > INT32_MAX) return af_set_error(AF_EINVAL, "af_candidates: bad nout");
    if (!isfinite(thresh)) return af_set_error(AF_EINVAL, "af_candidates: threshold not finite");
    af_widths_t w;
    if (int rc = af_check_widths(p, widths, nw, nout, &w)) return rc;
    return af_launch_candidates(d_best_snr, d_best_w, p->ndm, nout, w, thresh, sample0, d_out, cap, d_count,
                                (cudaStream_t)stream);
} catch (...) {
    return af_host_exception("af_candidates");
}

static bool cand_less_dt(const af_cand_t& a, const af_cand_t& b)
{
    if (a.dm_idx != b.dm_idx) return a.dm_idx < b.dm_idx;
    if (a.abs_sample != b.abs_sample) return a.abs_sample < b.abs_sample;
    return a.width < b.width;
}

extern "C" int af_cluster(af_plan_t p, af_cand_t* h_cands, int32_t n, double dm_tol, double toa_tol,
                          af_cand_t* h_out, int32_t* n_out)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (n < 0 || (n > 0 && (!h_cands || !h_out)) || !n_out) return af_set_error(AF_EINVAL, "af_cluster: bad args");
    for (int32_t i = 0; i < n; i++)
        if (h_cands[i].dm_idx < 0 || h_cands[i].dm_idx >= p->ndm)
            return af_set_error(AF_EINVAL, "af_cluster: dm_idx out of range");
    std::sort(h_cands, h_cands + n, cand_less_dt);
    std::vector<int32_t> order(n);
    for (int32_t i = 0; i < n; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        if (h_cands[a].snr != h_cands[b].snr) return h_cands[a].snr > h_cands[b].snr;
        return cand_less_dt(h_cands[a], h_cands[b]);
    });
    int32_t k = 0;
    for (int32_t i = 0; i < n; i++) {
        const af_cand_t& c = h_cands[order[i]];
        double dm = p->dms[c.dm_idx], toa = (double)c.abs_sample * p->tsamp;
        bool keep = true;
        for (int32_t j = 0; j < k && keep; j++) {
            if (fabs(p->dms[h_out[j].dm_idx] - dm) < dm_tol && fabs((double)h_out[j].abs_sample * p->tsamp - toa) < toa_tol)
                keep = false;
        }
        if (keep) h_out[k++] = c;
    }
    *n_out = k;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_cluster");
}

extern "C" int af_dedisperse_workspace_size(af_plan_t p, int64_t max_nsamp, size_t* bytes)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (!bytes) return af_set_error(AF_EINVAL, "af_dedisperse_workspace_size: NULL output");
    int64_t nout = 0;
    if (int rc = check_nout(p, max_nsamp, &nout)) return rc;
    *bytes = p->sb_nsub == 0 ? af_pairs_workspace(p, nout) : 0;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_dedisperse_workspace_size");
}

extern "C" int af_search_workspace_size(af_plan_t p, int64_t max_nsamp, int32_t cap, size_t* bytes)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (!bytes || cap < 1) return af_set_error(AF_EINVAL, "af_search_workspace_size: NULL output or cap < 1");
    int64_t nout = 0;
    if (int rc = check_nout(p, max_nsamp, &nout)) return rc;
    const size_t npl = (size_t)p->ndm * (size_t)nout;
    *bytes = (size_t)p->nchan * (size_t)max_nsamp + npl * 9 + (size_t)cap * sizeof(af_cand_t) + 16 +
             (p->sb_nsub == 0 ? af_pairs_workspace(p, nout) : 0);
    return AF_OK;
} catch (...) {
    return af_host_exception("af_search_workspace_size");
}

extern "C" int af_dedisperse_reserve(af_plan_t p, int64_t max_nsamp)
try {
    if (int rc = af_check_plan(p)) return rc;
    int64_t nout = 0;
    if (int rc = check_nout(p, max_nsamp, &nout)) return rc;
    return af_pairs_reserve(p, nout, false);
} catch (...) {
    return af_host_exception("af_dedisperse_reserve");
}

extern "C" int af_search_reserve(af_plan_t p, int64_t max_nsamp, int32_t cap)
try {
    if (int rc = af_check_plan(p)) return rc;
    int64_t nout = 0;
    if (int rc = check_nout(p, max_nsamp, &nout)) return rc;
    if (cap < 1) return af_set_error(AF_EINVAL, "af_search_reserve: cap must be >= 1");
    if (max_nsamp <= p->ws_nsamp && cap <= p->ws_cap) return AF_OK;
    free_search_ws(p);
    size_t nin = (size_t)p->nchan * (size_t)max_nsamp, npl = (size_t)p->ndm * (size_t)nout;
    cudaError_t e;
    if ((e = cudaMalloc(&p->ws_in, nin)) != cudaSuccess || (e = cudaMalloc(&p->ws_plane, npl * 4)) != cudaSuccess ||
        (e = cudaMalloc(&p->ws_snr, npl * 4)) != cudaSuccess || (e = cudaMalloc(&p->ws_bw, npl)) != cudaSuccess ||
        (e = cudaMalloc(&p->ws_cands, (size_t)cap * sizeof(af_cand_t))) != cudaSuccess ||
        (e = cudaMalloc(&p->ws_count, 16)) != cudaSuccess ||
        (e = cudaHostAlloc(&p->ws_host, 16 + (size_t)std::min(cap, kSearchStage) * sizeof(af_cand_t),
                           cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&p->ws_copy, cudaStreamNonBlocking)) != cudaSuccess) {
        free_search_ws(p);
        return af_cuda_check(e, "af_search_reserve");
    }
    for (cudaEvent_t& ev : p->ws_ev)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            free_search_ws(p);
            return af_cuda_check(e, "af_search_reserve: events");
        }
    p->ws_nsamp = max_nsamp;
    p->ws_cap = cap;
    p->ws_stage = std::min(cap, kSearchStage);
    search_bands(p);
    return af_pairs_reserve(p, nout, true);  // the group-row buffers, where that path applies
} catch (...) {
    return af_host_exception("af_search_reserve");
}

extern "C" int af_search_timing(af_plan_t p, int enable)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (enable && !p->ws_tev[0])
        for (cudaEvent_t& e : p->ws_tev)
            if (cudaError_t ce = cudaEventCreate(&e)) return af_cuda_check(ce, "af_search_timing");
    p->ws_timing = enable != 0;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_search_timing");
}

extern "C" int af_search_times(af_plan_t p, float* wait_ms, float* dedisp_ms, float* snr_ms)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (!p->ws_tev[0]) return af_set_error(AF_EINVAL, "af_search_times: timing was never enabled");
    float a = 0.f, b = 0.f, c = 0.f;
    AF_CUDA(cudaEventSynchronize(p->ws_tev[3]));
    AF_CUDA(cudaEventElapsedTime(&a, p->ws_tev[0], p->ws_tev[1]));
    AF_CUDA(cudaEventElapsedTime(&b, p->ws_tev[1], p->ws_tev[2]));
    AF_CUDA(cudaEventElapsedTime(&c, p->ws_tev[2], p->ws_tev[3]));
    if (wait_ms) *wait_ms = a;
    if (dedisp_ms) *dedisp_ms = b;
    if (snr_ms) *snr_ms = c;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_search_times");
}

extern "C" int af_search(af_plan_t p, const uint8_t* h_in, int64_t nsamp, const int32_t* widths, int nw,
                         float thresh, af_cand_t* h_out, int32_t cap, int32_t* h_count, void* stream)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (!h_in || !h_count || (cap > 0 && !h_out)) return af_set_error(AF_EINVAL, "af_search: NULL buffer");
    int64_t nout = 0;
    if (int rc = check_nout(p, nsamp, &nout)) return rc;
    if (nsamp > p->ws_nsamp || cap > p->ws_cap)
        return af_set_error(AF_ENOBUFS, "af_search: call af_search_reserve(nsamp >= %lld, cap >= %d) first",
                            (long long)nsamp, cap);
    af_widths_t w;
    if (int rc = af_check_widths(p, widths, nw, nout, &w)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const bool tm = p->ws_timing;
    if (tm) AF_CUDA(cudaEventRecord(p->ws_tev[0], s));
    if (af_dedisp_uses_pairs(p, nout)) {
        // Group rows: the outputs in growing time blocks (a small first one,
        // each next six times longer, at most the search layout's length);
        // each block's rows and tiles run as soon as its input columns (block
        // end + each channel band's largest delay) are in, overlapping the
        // rest of the copy.
        const int ly = p->pairs.lay[1].L > 0 ? 1 : 0;
        const int64_t tte = af_pair_tile_outputs();
        const std::vector<int64_t> blocks = af_search_block_tiles(nout, p->pairs.lay[ly].L / tte);
        AF_CUDA(cudaEventRecord(p->ws_ev[0], s));
        AF_CUDA(cudaStreamWaitEvent(p->ws_copy, p->ws_ev[0], 0));
        AF_CUDA(cudaMemsetAsync(p->d_stats, 0, (size_t)p->ndm * sizeof(af_rowstats_t), s));
        int64_t col[kSearchBands] = {}, T0 = 0;
        for (size_t k = 0; k < blocks.size(); k++) {
            const int64_t L = blocks[k] * tte;
            if (int rc = search_copy_upto(p, h_in, nsamp, T0 + L, T0 + L >= nout, col)) return rc;
            cudaEvent_t ev = p->ws_ev[k % 4];  // an event is reused once the stream has waited on it
            AF_CUDA(cudaEventRecord(ev, p->ws_copy));
            AF_CUDA(cudaStreamWaitEvent(s, ev, 0));
            if (tm && k == 0) AF_CUDA(cudaEventRecord(p->ws_tev[1], s));
            if (int rc = af_launch_pairs_block(p, p->ws_in, nsamp, nout, p->ws_plane, p->d_stats, s, ly, T0, nullptr, L))
                return rc;
            T0 += L;
        }
    } else if (af_dedisp_uses_tiles(p)) {
        // The input arrives in time segments on the copy stream; each segment's
        // output tiles are dedispersed as soon as their columns (and each
        // channel band's delay halo after them) are in, overlapping the rest
        // of the copy.
        const int64_t tte = af_dedisp_tile_outputs();
        const unsigned tiles = (unsigned)((nout + tte - 1) / tte);
        const unsigned K = tiles < 4u ? tiles : 4u;
        AF_CUDA(cudaEventRecord(p->ws_ev[0], s));  // copies follow the caller's earlier work on s
        AF_CUDA(cudaStreamWaitEvent(p->ws_copy, p->ws_ev[0], 0));
        AF_CUDA(cudaMemsetAsync(p->d_stats, 0, (size_t)p->ndm * sizeof(af_rowstats_t), s));
        int64_t col[kSearchBands] = {};
        for (unsigned k = 0; k < K; k++) {
            const unsigned tb = tiles * k / K, te = tiles * (k + 1) / K;
            if (int rc = search_copy_upto(p, h_in, nsamp, (int64_t)te * tte, k + 1 == K, col)) return rc;
            AF_CUDA(cudaEventRecord(p->ws_ev[k], p->ws_copy));
            AF_CUDA(cudaStreamWaitEvent(s, p->ws_ev[k], 0));
            if (tm && k == 0) AF_CUDA(cudaEventRecord(p->ws_tev[1], s));
            if (int rc = af_launch_dedisperse_tiles(p, p->ws_in, nsamp, nout, p->ws_plane, p->d_stats, s, tb, te))
                return rc;
        }
    } else {
        AF_CUDA(cudaMemcpyAsync(p->ws_in, h_in, (size_t)p->nchan * nsamp, cudaMemcpyHostToDevice, s));
        if (tm) AF_CUDA(cudaEventRecord(p->ws_tev[1], s));
        if (int rc = af_launch_dedisperse(p, p->ws_in, nsamp, nout, p->ws_plane, p->d_stats, s)) return rc;
    }
    if (tm) AF_CUDA(cudaEventRecord(p->ws_tev[2], s));
    if (int rc = af_launch_boxcar(p->ws_plane, p->ndm, nout, p->d_stats, w, p->d_rowconst, p->ws_snr, p->ws_bw, s))
        return rc;
    if (int rc = af_launch_candidates(p->ws_snr, p->ws_bw, p->ndm, nout, w, thresh, 0, p->ws_cands, cap,
                                      p->ws_count, s))
        return rc;
    if (tm) AF_CUDA(cudaEventRecord(p->ws_tev[3], s));
    // One wait in the usual case: the count, the error flag and the first
    // ws_stage candidates come back together into pinned memory; only a
    // larger candidate list takes a second copy.
    int32_t* hs = p->ws_host;
    af_cand_t* hc = reinterpret_cast<af_cand_t*>(hs + 4);
    const int32_t stage = std::min(cap, p->ws_stage);
    AF_CUDA(cudaMemcpyAsync(hs, p->ws_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AF_CUDA(cudaMemcpyAsync(hs + 1, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (stage > 0)
        AF_CUDA(cudaMemcpyAsync(hc, p->ws_cands, (size_t)stage * sizeof(af_cand_t), cudaMemcpyDeviceToHost, s));
    AF_CUDA(cudaStreamSynchronize(s));
    const int32_t total = hs[0];
    if (hs[1]) {
        AF_CUDA(cudaMemsetAsync(p->d_err, 0, sizeof(int), s));
        return af_set_error(AF_ETIMEOUT, "af_search: a kernel's bounded wait for an asynchronous copy ran out");
    }
    int32_t ncopy = total < cap ? total : cap;
    if (ncopy > 0) {
        if (ncopy <= stage) {
            memcpy(h_out, hc, (size_t)ncopy * sizeof(af_cand_t));
        } else {
            AF_CUDA(cudaMemcpyAsync(h_out, p->ws_cands, (size_t)ncopy * sizeof(af_cand_t), cudaMemcpyDeviceToHost,
                                    s));
            AF_CUDA(cudaStreamSynchronize(s));
        }
        std::sort(h_out, h_out + ncopy, cand_less_dt);
    }
    *h_count = total;
    if (total > cap) return af_set_error(AF_EOVERFLOW, "af_search: %d candidates, capacity %d", total, cap);
    return AF_OK;
} catch (...) {
    return af_host_exception("af_search");
}
