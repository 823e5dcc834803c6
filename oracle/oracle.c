/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle for the single-pulse
 * search hot path (ASTROFLOW, arXiv 2511.02328).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so, which
 * only the test-suite, the smoke check and the CPU-baseline leg of bench.py
 * load.  It shares no code, header, table or constant with the CUDA library
 * (paper_2511_02328_gb300/csrc); neither side includes or links the other.
 *
 * Every function below is the plain definition written out as loops, in
 * double precision wherever floating point appears, with the section /
 * equation of the paper it follows.  Where the paper is silent the reading
 * used is stated next to the code ("Reading: ...").
 *
 * Pins: every function here is checked by the -m "not gpu" tests against
 * something other than itself (exact rational arithmetic, brute force in pure
 * Python, closed forms, invariants, injected-pulse recovery).
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* Dispersion constant of Eq. (KDM), Sec. 2.3.  The paper prints the unit as
 * "ms MHz^2 pc^-1 cm^3"; with f in MHz the value 4.148808e3 gives SECONDS
 * (DM 1000 between 1000 and 1500 MHz is then 2.305 s, the physical value).
 * Reading: unit = s.                                                       */
static const double ORACLE_K_DM = 4.148808e3;

/* Reading (paper silent): channel c of nchan covers [f_lo + c*df, f_lo+(c+1)*df]
 * with df = (f_hi - f_lo)/nchan, and its frequency is the centre.  f_hi < f_lo
 * describes a descending band (channel 0 highest).                          */
double oracle_chan_freq(int c, int nchan, double f_lo, double f_hi)
{
    double df = (f_hi - f_lo) / (double)nchan;
    return f_lo + ((double)c + 0.5) * df;
}

/* Reading: f_ref = the top edge of the band (TOA "referenced to the top of the
 * band", Sec. 2; matching "referenced to 1500 MHz", Sec. 4.2).             */
double oracle_ref_freq(double f_lo, double f_hi)
{
    return f_lo > f_hi ? f_lo : f_hi;
}

/* Integer delay table, Eq. (coarse_delay) with the DM grid given explicitly:
 *     D[d][c] = round( K*DM_d/t_samp * (1/f_c^2 - 1/f_ref^2) )
 * Reading: round = half away from zero (llround), evaluated in IEEE double in
 * exactly this order, with no fused multiply-add:
 *     a = (K*dm)/tsamp ; b = 1/(fc*fc) - 1/(fr*fr) ; D = llround(a*b).
 * Returns 0 on success, -1 on invalid arguments, -2 if a delay overflows int32. */
int oracle_delay_table(int nchan, double f_lo, double f_hi, double tsamp,
                       const double* dm, int ndm, int32_t* D)
{
    if (nchan <= 0 || ndm <= 0 || !(tsamp > 0.0) || !(f_lo > 0.0) || !(f_hi > 0.0) || f_lo == f_hi)
        return -1;
    double fr = oracle_ref_freq(f_lo, f_hi);
    for (int d = 0; d < ndm; d++) {
        if (!(dm[d] >= 0.0) || !isfinite(dm[d]))
            return -1;
        double a = (ORACLE_K_DM * dm[d]) / tsamp;
        for (int c = 0; c < nchan; c++) {
            double fc = oracle_chan_freq(c, nchan, f_lo, f_hi);
            double b = 1.0 / (fc * fc) - 1.0 / (fr * fr);
            double x = a * b;
            if (!(x < 2147483647.0))
                return -2;
            D[(int64_t)d * nchan + c] = (int32_t)llround(x);
        }
    }
    return 0;
}

/* Largest entry of a delay table. */
int32_t oracle_dmax(const int32_t* D, int ndm, int nchan)
{
    int32_t m = 0;
    for (int64_t i = 0; i < (int64_t)ndm * nchan; i++)
        if (D[i] > m) m = D[i];
    return m;
}

/* Brute-force incoherent dedispersion, Sec. 2.3 (the O(N_DM N_t N_f) method
 * that the paper's subband scheme approximates):
 *     Y[d][t] = sum_c X[c][t + D[d][c]],   0 <= t < nout
 * X is uint8 [nchan][nsamp] (channel-major), Y is int32 [ndm][nout].
 * Reading: nout = nsamp - Dmax of the whole table, so every term is inside
 * the data and no zero padding is needed (the paper truncates by the DM delay,
 * Sec. 3).  The caller passes nout; every delay must satisfy D + nout <= nsamp.
 * Loop order d, c, t; OpenMP over DM rows only.                            */
/* Threads of the OpenMP team that the parallel loops below run on (not part
 * of the method: reported beside the oracle's timings). */
int oracle_threads(void)
{
    int n = 1;
    #pragma omp parallel
    {
        #pragma omp single
        n = omp_get_num_threads();
    }
    return n;
}

void oracle_dedisperse(const uint8_t* X, int nchan, int64_t nsamp,
                       const int32_t* D, int ndm, int64_t nout, int32_t* Y)
{
    (void)nsamp;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int d = 0; d < ndm; d++) {
        int32_t* y = Y + (int64_t)d * nout;
        for (int64_t t = 0; t < nout; t++)
            y[t] = 0;
        for (int c = 0; c < nchan; c++) {
            const uint8_t* x = X + (int64_t)c * nsamp + D[(int64_t)d * nchan + c];
            for (int64_t t = 0; t < nout; t++)
                y[t] += (int32_t)x[t];
        }
    }
}

/* Row statistics (reading; the paper gives no normalisation):
 *     S_d = sum_t Y[d][t],  Q_d = sum_t Y[d][t]^2   (exact, int64)         */
void oracle_rowstats(const int32_t* Y, int ndm, int64_t nout, int64_t* S, int64_t* Q)
{
    #pragma omp parallel for schedule(static)
    for (int d = 0; d < ndm; d++) {
        int64_t s = 0, q = 0;
        const int32_t* y = Y + (int64_t)d * nout;
        for (int64_t t = 0; t < nout; t++) {
            s += y[t];
            q += (int64_t)y[t] * y[t];
        }
        S[d] = s;
        Q[d] = q;
    }
}

/* Population standard deviation of a row from its exact sums:
 *     sigma^2 = (nout*Q - S^2) / nout^2   (numerator exact in 128 bits)    */
double oracle_row_sigma(int64_t S, int64_t Q, int64_t nout)
{
    __int128 num = (__int128)nout * Q - (__int128)S * S;
    double var = (double)num / ((double)nout * (double)nout);
    return var > 0.0 ? sqrt(var) : 0.0;
}

/* Boxcar matched filter and S/N, step (iii) of the standard workflow (Sec. 1);
 * definitions are readings, the paper names the step only:
 *     B_w[t] = sum_{k=t}^{t+w-1} Y[d][k]          (window leading edge at t)
 *     snr_w  = (nout*B_w - w*S_d) / (nout * sigma_d * sqrt(w))
 * which is (B_w - w*mu)/(sigma*sqrt(w)) with mu = S/nout.  The numerator is
 * exact in 128-bit integers.  A width with t + w > nout is not valid at t.
 * best_snr[d][t] = max over valid widths, ties to the smaller width (widths
 * must be strictly ascending); best_w[d][t] = index into widths of the max,
 * or -1 (with best_snr = -inf) when no width is valid.  sigma = 0 gives snr 0. */
void oracle_boxcar_snr(const int32_t* Y, int ndm, int64_t nout,
                       const int32_t* widths, int nw,
                       double* best_snr, int32_t* best_w)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int d = 0; d < ndm; d++) {
        const int32_t* y = Y + (int64_t)d * nout;
        int64_t S = 0, Q = 0;
        for (int64_t t = 0; t < nout; t++) {
            S += y[t];
            Q += (int64_t)y[t] * y[t];
        }
        double sigma = oracle_row_sigma(S, Q, nout);
        for (int64_t t = 0; t < nout; t++) {
            double best = -INFINITY;
            int32_t bi = -1;
            for (int i = 0; i < nw; i++) {
                int64_t w = widths[i];
                if (t + w > nout)
                    continue;
                int64_t B = 0;
                for (int64_t k = t; k < t + w; k++)
                    B += y[k];
                double snr;
                if (sigma > 0.0) {
                    __int128 num = (__int128)nout * B - (__int128)w * S;
                    snr = (double)num / ((double)nout * sigma * sqrt((double)w));
                } else {
                    snr = 0.0;
                }
                if (snr > best) {
                    best = snr;
                    bi = i;
                }
            }
            best_snr[(int64_t)d * nout + t] = best;
            best_w[(int64_t)d * nout + t] = bi;
        }
    }
}

/* Candidate record produced by oracle_peaks (same field meaning as the
 * library's, declared independently). */
typedef struct {
    int32_t dm_idx;
    int32_t t;
    int32_t width;
    double snr;
} oracle_cand_t;

/* Threshold + local-maximum test (reading; the paper thresholds "by S/N and DM
 * criteria", Sec. 2):  (d,t) is a candidate iff best_snr[d][t] >= thresh and,
 * with w = widths[best_w[d][t]],
 *     best_snr[d][t] >  best_snr[d][u]  for t-w <= u < t,
 *     best_snr[d][t] >= best_snr[d][u]  for t < u <= t+w   (ties: earliest t).
 * Output in (d, t) order.  Returns the total number of candidates, of which at
 * most cap are written.                                                    */
int64_t oracle_peaks(const double* best_snr, const int32_t* best_w, int ndm, int64_t nout,
                     const int32_t* widths, double thresh, oracle_cand_t* out, int64_t cap)
{
    int64_t n = 0;
    for (int d = 0; d < ndm; d++) {
        const double* s = best_snr + (int64_t)d * nout;
        const int32_t* bw = best_w + (int64_t)d * nout;
        for (int64_t t = 0; t < nout; t++) {
            if (!(s[t] >= thresh) || bw[t] < 0)
                continue;
            int64_t w = widths[bw[t]];
            int peak = 1;
            for (int64_t u = t - w; u <= t + w && peak; u++) {
                if (u < 0 || u >= nout || u == t)
                    continue;
                if (u < t && !(s[t] > s[u])) peak = 0;
                if (u > t && !(s[t] >= s[u])) peak = 0;
            }
            if (!peak)
                continue;
            if (n < cap) {
                out[n].dm_idx = d;
                out[n].t = (int32_t)t;
                out[n].width = (int32_t)w;
                out[n].snr = s[t];
            }
            n++;
        }
    }
    return n;
}

/* ======================================================================
 * Two-stage subband dedispersion (Sec. 2.3, Eqs. stage1, residual, stage2).
 * ====================================================================== */

/* Subband partition.  Reading (the paper only says the channels are
 * partitioned into subbands): nsub contiguous groups of as-equal-as-possible
 * size, subband s = channels [floor(s*nchan/nsub), floor((s+1)*nchan/nsub)).
 * first[] has nsub+1 entries.  Returns 0, or -1 on invalid arguments.       */
int oracle_subband_first(int nchan, int nsub, int32_t* first)
{
    if (nchan <= 0 || nsub <= 0 || nsub > nchan)
        return -1;
    for (int s = 0; s <= nsub; s++)
        first[s] = (int32_t)(((int64_t)s * nchan) / nsub);
    return 0;
}

static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Representative frequency F_s of the channels [c0, c1) (Sec. 2.3: "the
 * median or a 1/f^2-weighted center").  Readings:
 *   mode 0: median of the channel-centre frequencies (mean of the two middle
 *           values when the count is even);
 *   mode 1: the frequency whose 1/F^2 equals the mean of 1/f_c^2 over the
 *           subband, F = (mean 1/f_c^2)^(-1/2)  (the centre of the quantity
 *           the delay is linear in).
 * Returns a negative value on invalid arguments.                            */
double oracle_subband_freq(int nchan, double f_lo, double f_hi, int c0, int c1, int mode)
{
    int n = c1 - c0;
    if (n <= 0 || c0 < 0 || c1 > nchan)
        return -1.0;
    if (mode == 0) {
        double* f = (double*)malloc(sizeof(double) * n);
        if (!f)
            return -1.0;
        for (int i = 0; i < n; i++)
            f[i] = oracle_chan_freq(c0 + i, nchan, f_lo, f_hi);
        qsort(f, n, sizeof(double), cmp_double);
        double med = (n % 2) ? f[n / 2] : 0.5 * (f[n / 2 - 1] + f[n / 2]);
        free(f);
        return med;
    }
    if (mode == 1) {
        double acc = 0.0;
        for (int c = c0; c < c1; c++) {
            double fc = oracle_chan_freq(c, nchan, f_lo, f_hi);
            acc += 1.0 / (fc * fc);
        }
        return 1.0 / sqrt(acc / (double)n);
    }
    return -1.0;
}

/* Residual shift table, Eq. (residual).  The fine DM list dm[0..ndm) is
 * grouped N0 at a time: j(m) = floor(m/N0), coarse DM_j = dm[j*N0] (for an
 * evenly spaced list this is DM_low + j*N0*dDM, the paper's coarse grid), and
 *     R[m][s] = round( K*(dm[m] - DM_j(m))/t_samp * (1/F_s^2 - 1/f_ref^2) )
 * with the rounding and operation order of Eq. (coarse_delay) (llround of
 * a*b, a = K*dDM/tsamp, b = 1/(F*F) - 1/(fr*fr)).  Reading: the list must be
 * non-decreasing, so every residual DM and shift is >= 0.
 * Returns 0, -1 on invalid arguments, -2 on int32 overflow.                 */
int oracle_subband_residuals(int nchan, double f_lo, double f_hi, double tsamp, const double* dm, int ndm,
                             int n0, int nsub, int mode, int32_t* R)
{
    if (nchan <= 0 || ndm <= 0 || n0 <= 0 || nsub <= 0 || nsub > nchan || !(tsamp > 0.0))
        return -1;
    for (int m = 1; m < ndm; m++)
        if (!(dm[m] >= dm[m - 1]))
            return -1;
    int32_t* first = (int32_t*)malloc(sizeof(int32_t) * (nsub + 1));
    if (!first)
        return -1;
    oracle_subband_first(nchan, nsub, first);
    double fr = oracle_ref_freq(f_lo, f_hi);
    int rc = 0;
    for (int s = 0; s < nsub && rc == 0; s++) {
        double F = oracle_subband_freq(nchan, f_lo, f_hi, first[s], first[s + 1], mode);
        if (!(F > 0.0)) {
            rc = -1;
            break;
        }
        double b = 1.0 / (F * F) - 1.0 / (fr * fr);
        for (int m = 0; m < ndm; m++) {
            double ddm = dm[m] - dm[(m / n0) * n0];
            double a = (ORACLE_K_DM * ddm) / tsamp;
            double x = a * b;
            if (!(x < 2147483647.0)) {
                rc = -2;
                break;
            }
            R[(int64_t)m * nsub + s] = (int32_t)llround(x);
        }
    }
    free(first);
    return rc;
}

/* Two-stage subband dedispersion, Eqs. (stage1) and (stage2), Sec. 2.3.
 *   Dc     int32 [ncoarse][nchan]: delays of the coarse DMs, Eq. (coarse_delay)
 *   first  int32 [nsub+1]: the partition;  R int32 [ndm][nsub]: Eq. (residual)
 * Stage 1, for every coarse DM j and subband s (X is zero outside the data):
 *     I(j,s,u) = sum_{c in C_s} X(c, u + D[j][c]),  0 <= u < nout + max_{m in j, s} R[m][s]
 * Stage 2, for every fine DM m (j = floor(m/N0)):
 *     Y(m,v) = sum_s I(j, s, v + R[m][s]),  0 <= v < nout.
 * Reading: no time blocking (the paper's block length L only bounds memory;
 * with nout = nsamp - max_{m,c}(D[j(m)][c] + R[m][s(c)]) every block gives
 * the same values), so the whole time axis is one block.  The caller passes
 * nout.  Stage 1 is evaluated per coarse DM (I of one j at a time).         */
int oracle_subband_dedisperse(const uint8_t* X, int nchan, int64_t nsamp, const int32_t* Dc, int ncoarse,
                              const int32_t* first, int nsub, const int32_t* R, int ndm, int n0, int64_t nout,
                              int32_t* Y)
{
    if (n0 <= 0 || ncoarse != (ndm + n0 - 1) / n0 || nout <= 0)
        return -1;
    for (int j = 0; j < ncoarse; j++) {
        int m_lo = j * n0, m_hi = (j + 1) * n0 < ndm ? (j + 1) * n0 : ndm;
        int32_t rmax = 0;
        for (int m = m_lo; m < m_hi; m++)
            for (int s = 0; s < nsub; s++)
                if (R[(int64_t)m * nsub + s] > rmax) rmax = R[(int64_t)m * nsub + s];
        int64_t li = nout + rmax;
        int32_t* I = (int32_t*)calloc((size_t)nsub * li, sizeof(int32_t));
        if (!I)
            return -2;
        /* Stage 1 */
        #pragma omp parallel for schedule(dynamic, 1)
        for (int s = 0; s < nsub; s++) {
            int32_t* Is = I + (int64_t)s * li;
            for (int c = first[s]; c < first[s + 1]; c++) {
                int64_t d = Dc[(int64_t)j * nchan + c];
                const uint8_t* x = X + (int64_t)c * nsamp;
                for (int64_t u = 0; u < li; u++) {
                    int64_t t = u + d;
                    if (t >= 0 && t < nsamp)
                        Is[u] += (int32_t)x[t];
                }
            }
        }
        /* Stage 2 */
        #pragma omp parallel for schedule(dynamic, 1)
        for (int m = m_lo; m < m_hi; m++) {
            int32_t* y = Y + (int64_t)m * nout;
            for (int64_t v = 0; v < nout; v++)
                y[v] = 0;
            for (int s = 0; s < nsub; s++) {
                const int32_t* Is = I + (int64_t)s * li;
                int64_t r = R[(int64_t)m * nsub + s];
                for (int64_t v = 0; v < nout; v++) {
                    int64_t u = v + r;
                    if (u >= 0 && u < li)
                        y[v] += Is[u];
                }
            }
        }
        free(I);
    }
    return 0;
}

/* ======================================================================
 * Square-law time downsampling (Sec. 2.2, "Downsampling and Subband
 * Combination").
 * ====================================================================== */

/* For each channel and each bin k of D consecutive samples (the last bin
 * holds the remaining nsamp - (nout-1)*D samples, nout = ceil(nsamp/D), the
 * paper's N_t = ceil(N_t/D)), with S the sum of the bin's N samples:
 *     out = min( V * sqrt(S) / sqrt(N*V), V ) = min( sqrt(V*S/N), V ).
 * Reading (the paper does not say how the value becomes an integer of the
 * chosen bit width): round to nearest, halves up, evaluated exactly in integer
 * arithmetic: round(sqrt(q)) = floor((isqrt(floor(4q)) + 1) / 2) for q >= 0,
 * with 4q = 4*V*S/N.  V = vmax (255 for 8-bit data).
 * X uint8 [nchan][nsamp]; out uint8 [nchan][ceil(nsamp/D)].
 * Returns 0, or -1 on invalid arguments.                                     */
static uint64_t isqrt_u64(uint64_t x)
{
    uint64_t r = 0, bit = (uint64_t)1 << 62;
    while (bit > x) bit >>= 2;
    while (bit) {
        if (x >= r + bit) {
            x -= r + bit;
            r = (r >> 1) + bit;
        } else {
            r >>= 1;
        }
        bit >>= 2;
    }
    return r;
}

int oracle_downsample_sqlaw(const uint8_t* X, int nchan, int64_t nsamp, int D, int vmax, uint8_t* out)
{
    if (nchan <= 0 || nsamp <= 0 || D <= 0 || vmax <= 0 || vmax > 255)
        return -1;
    int64_t nout = (nsamp + D - 1) / D;
    for (int c = 0; c < nchan; c++) {
        const uint8_t* x = X + (int64_t)c * nsamp;
        for (int64_t k = 0; k < nout; k++) {
            int64_t t0 = k * D, t1 = t0 + D < nsamp ? t0 + D : nsamp;
            uint64_t S = 0, N = (uint64_t)(t1 - t0);
            for (int64_t t = t0; t < t1; t++)
                S += x[t];
            uint64_t r = isqrt_u64((4u * (uint64_t)vmax * S) / N);
            uint64_t v = (r + 1) / 2;
            out[(int64_t)c * nout + k] = (uint8_t)(v < (uint64_t)vmax ? v : (uint64_t)vmax);
        }
    }
    return 0;
}

/* ======================================================================
 * Zero-DM filter and robust (median/MAD) S/N normalisation (Sec. 2.1 RFI
 * mitigation; Sec. 4.4 names zero-DM filtering as the remedy for impulsive
 * broadband RFI).
 * ====================================================================== */

/* Zero-DM filter: the mean over channels at each time sample (the DM = 0
 * time series divided by nchan) is removed from every channel.  Readings (the
 * paper gives no formula): the mean is rounded to nearest, halves up, exactly,
 *     q[t] = floor((2 * sum_c X[c][t] + nchan) / (2 * nchan)),
 * and the 8-bit result is re-centred on mid-scale and clipped:
 *     X'[c][t] = min(255, max(0, X[c][t] - q[t] + 128)).
 * X and out uint8 [nchan][nsamp] (out may equal X).  Returns 0 or -1.       */
int oracle_zerodm(const uint8_t* X, int nchan, int64_t nsamp, uint8_t* out)
{
    if (nchan <= 0 || nsamp <= 0)
        return -1;
    int64_t* q = (int64_t*)malloc(sizeof(int64_t) * nsamp);
    if (!q)
        return -1;
    for (int64_t t = 0; t < nsamp; t++) {
        int64_t s = 0;
        for (int c = 0; c < nchan; c++)
            s += X[(int64_t)c * nsamp + t];
        q[t] = (2 * s + nchan) / (2 * (int64_t)nchan);
    }
    for (int c = 0; c < nchan; c++)
        for (int64_t t = 0; t < nsamp; t++) {
            int64_t v = (int64_t)X[(int64_t)c * nsamp + t] - q[t] + 128;
            out[(int64_t)c * nsamp + t] = (uint8_t)(v < 0 ? 0 : v > 255 ? 255 : v);
        }
    free(q);
    return 0;
}

static int cmp_i64(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

/* Robust location and scale of each plane row (reading of the robust S/N
 * normalisation):  med_d = the lower median of the row (element (nout-1)/2 of
 * the sorted row), mad_d = the lower median of |Y[d][t] - med_d|.  Both are
 * integers.  The S/N scale is sigma_d = 1.482602218505602 * mad_d (the MAD of
 * a normal distribution is sigma / 1.4826...).                              */
void oracle_row_robust(const int32_t* Y, int ndm, int64_t nout, int64_t* med, int64_t* mad)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int d = 0; d < ndm; d++) {
        int64_t* v = (int64_t*)malloc(sizeof(int64_t) * nout);
        const int32_t* y = Y + (int64_t)d * nout;
        for (int64_t t = 0; t < nout; t++)
            v[t] = y[t];
        qsort(v, nout, sizeof(int64_t), cmp_i64);
        int64_t m = v[(nout - 1) / 2];
        for (int64_t t = 0; t < nout; t++)
            v[t] = y[t] >= m ? y[t] - m : m - y[t];
        qsort(v, nout, sizeof(int64_t), cmp_i64);
        med[d] = m;
        mad[d] = v[(nout - 1) / 2];
        free(v);
    }
}

/* Boxcar S/N with an explicit location mu_d and scale sigma_d per row:
 *     snr_w = (B_w - w*mu_d) / (sigma_d * sqrt(w))
 * with the window, validity and tie rules of oracle_boxcar_snr; sigma_d = 0
 * gives snr 0.  (mu = S/nout and sigma = the population deviation give
 * oracle_boxcar_snr; mu = med and sigma = 1.4826*mad the robust S/N.)      */
void oracle_boxcar_snr_norm(const int32_t* Y, int ndm, int64_t nout, const int32_t* widths, int nw,
                            const double* mu, const double* sigma, double* best_snr, int32_t* best_w)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int d = 0; d < ndm; d++) {
        const int32_t* y = Y + (int64_t)d * nout;
        for (int64_t t = 0; t < nout; t++) {
            double best = -INFINITY;
            int32_t bi = -1;
            for (int i = 0; i < nw; i++) {
                int64_t w = widths[i];
                if (t + w > nout)
                    continue;
                int64_t B = 0;
                for (int64_t k = t; k < t + w; k++)
                    B += y[k];
                double snr = sigma[d] > 0.0 ? ((double)B - (double)w * mu[d]) / (sigma[d] * sqrt((double)w)) : 0.0;
                if (snr > best) {
                    best = snr;
                    bi = i;
                }
            }
            best_snr[(int64_t)d * nout + t] = best;
            best_w[(int64_t)d * nout + t] = bi;
        }
    }
}
