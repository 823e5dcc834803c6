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
