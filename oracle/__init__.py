"""CPU oracle for the single-pulse search hot path (ASTROFLOW, arXiv 2511.02328).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import this package.  It shares
no code with the CUDA library and never calls it.

The heavy loops live in oracle.c (plain C, fp64, OpenMP over DM rows); this
module loads it with ctypes and adds numpy-friendly wrappers.  The pure-Python
brute force for tiny inputs is in oracle.brute, the candidate clustering and
matching rule in oracle.nms, the cut-out and CNN oracles in oracle.cutout and
oracle.cnn, the DM-time slice gridding in oracle.grid.
"""
import ctypes
import os

import numpy as np

from .build import build_oracle

_lib = None


class OracleCand(ctypes.Structure):
    _fields_ = [("dm_idx", ctypes.c_int32), ("t", ctypes.c_int32),
                ("width", ctypes.c_int32), ("snr", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = ctypes.CDLL(path)
        L.oracle_chan_freq.restype = ctypes.c_double
        L.oracle_chan_freq.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.oracle_ref_freq.restype = ctypes.c_double
        L.oracle_ref_freq.argtypes = [ctypes.c_double, ctypes.c_double]
        L.oracle_delay_table.restype = ctypes.c_int
        L.oracle_delay_table.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        L.oracle_dmax.restype = ctypes.c_int32
        L.oracle_dmax.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.oracle_dedisperse.restype = None
        L.oracle_threads.restype = ctypes.c_int
        L.oracle_threads.argtypes = []
        L.oracle_dedisperse.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_int64, ctypes.c_void_p]
        L.oracle_rowstats.restype = None
        L.oracle_rowstats.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_void_p]
        L.oracle_row_sigma.restype = ctypes.c_double
        L.oracle_row_sigma.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
        L.oracle_boxcar_snr.restype = None
        L.oracle_boxcar_snr.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_peaks.restype = ctypes.c_int64
        L.oracle_peaks.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                   ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64]
        L.oracle_subband_first.restype = ctypes.c_int
        L.oracle_subband_first.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        L.oracle_subband_freq.restype = ctypes.c_double
        L.oracle_subband_freq.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int]
        L.oracle_subband_residuals.restype = ctypes.c_int
        L.oracle_subband_residuals.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_void_p]
        L.oracle_subband_dedisperse.restype = ctypes.c_int
        L.oracle_subband_dedisperse.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                                ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p]
        L.oracle_downsample_sqlaw.restype = ctypes.c_int
        L.oracle_downsample_sqlaw.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_void_p]
        L.oracle_zerodm.restype = ctypes.c_int
        L.oracle_zerodm.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p]
        L.oracle_row_robust.restype = None
        L.oracle_row_robust.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_void_p]
        L.oracle_boxcar_snr_norm.restype = None
        L.oracle_boxcar_snr_norm.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                             ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def chan_freqs(nchan, f_lo, f_hi):
    """Channel-centre frequencies in MHz (reading: centres), via the C oracle."""
    L = lib()
    return np.array([L.oracle_chan_freq(c, nchan, f_lo, f_hi) for c in range(nchan)])


def delay_table(nchan, f_lo, f_hi, tsamp, dms):
    """int32 [ndm][nchan] integer delays, Eq. (coarse_delay) (Sec. 2.3)."""
    dms = np.ascontiguousarray(dms, dtype=np.float64)
    D = np.empty((dms.size, nchan), dtype=np.int32)
    rc = lib().oracle_delay_table(nchan, f_lo, f_hi, tsamp, _ptr(dms), dms.size, _ptr(D))
    if rc != 0:
        raise ValueError("oracle_delay_table failed (%d)" % rc)
    return D


def dedisperse(X, D, nout=None):
    """Brute-force plane Y[d][t] = sum_c X[c][t + D[d][c]] (Sec. 2.3), int32."""
    X = np.ascontiguousarray(X, dtype=np.uint8)
    D = np.ascontiguousarray(D, dtype=np.int32)
    nchan, nsamp = X.shape
    ndm = D.shape[0]
    if D.shape[1] != nchan:
        raise ValueError("delay table / data channel mismatch")
    if nout is None:
        nout = nsamp - int(D.max())
    if nout <= 0 or int(D.max()) + nout > nsamp or int(D.min()) < 0:
        raise ValueError("nout out of range")
    Y = np.empty((ndm, nout), dtype=np.int32)
    lib().oracle_dedisperse(_ptr(X), nchan, nsamp, _ptr(D), ndm, nout, _ptr(Y))
    return Y


def rowstats(Y):
    Y = np.ascontiguousarray(Y, dtype=np.int32)
    ndm, nout = Y.shape
    S = np.empty(ndm, dtype=np.int64)
    Q = np.empty(ndm, dtype=np.int64)
    lib().oracle_rowstats(_ptr(Y), ndm, nout, _ptr(S), _ptr(Q))
    return S, Q


def row_sigma(S, Q, nout):
    return lib().oracle_row_sigma(int(S), int(Q), int(nout))


def boxcar_snr(Y, widths):
    """(best_snr float64 [ndm][nout], best_w int32 index [ndm][nout])."""
    Y = np.ascontiguousarray(Y, dtype=np.int32)
    widths = np.ascontiguousarray(widths, dtype=np.int32)
    if widths.size == 0 or np.any(np.diff(widths) <= 0) or widths[0] < 1:
        raise ValueError("widths must be strictly ascending and >= 1")
    ndm, nout = Y.shape
    snr = np.empty((ndm, nout), dtype=np.float64)
    bw = np.empty((ndm, nout), dtype=np.int32)
    lib().oracle_boxcar_snr(_ptr(Y), ndm, nout, _ptr(widths), widths.size, _ptr(snr), _ptr(bw))
    return snr, bw


def peaks(best_snr, best_w, widths, thresh, cap=1 << 22):
    """List of (dm_idx, t, width, snr) in (d, t) order, and the total count."""
    best_snr = np.ascontiguousarray(best_snr, dtype=np.float64)
    best_w = np.ascontiguousarray(best_w, dtype=np.int32)
    widths = np.ascontiguousarray(widths, dtype=np.int32)
    ndm, nout = best_snr.shape
    out = (OracleCand * cap)()
    n = lib().oracle_peaks(_ptr(best_snr), _ptr(best_w), ndm, nout, _ptr(widths), float(thresh),
                           ctypes.cast(out, ctypes.c_void_p), cap)
    res = [(out[i].dm_idx, out[i].t, out[i].width, out[i].snr) for i in range(min(n, cap))]
    return res, int(n)


def search(X, D, widths, thresh):
    """Whole plain search on the CPU: plane, S/N, candidates."""
    Y = dedisperse(X, D)
    snr, bw = boxcar_snr(Y, widths)
    cands, n = peaks(snr, bw, widths, thresh)
    return Y, snr, bw, cands


def injection_offsets(nchan, f_lo, f_hi, tsamp, dm, t0):
    """Per-channel start sample of a pulse that arrives at f_ref at sample t0
    with dispersion measure dm: t0 + D_inj[c], where D_inj uses the same
    rounding as Eq. (coarse_delay).  Used to build injected test inputs."""
    D = delay_table(nchan, f_lo, f_hi, tsamp, [dm])[0]
    return (np.int64(t0) + D.astype(np.int64))


FS_MEDIAN = 0   # representative frequency: median of the channel centres
FS_INVSQ = 1    # representative frequency: 1/F^2 = mean of 1/f_c^2


def subband_first(nchan, nsub):
    """Partition of the channels into nsub contiguous subbands (Sec. 2.3):
    int32 [nsub+1], subband s = channels [first[s], first[s+1])."""
    first = np.empty(nsub + 1, dtype=np.int32)
    if lib().oracle_subband_first(nchan, nsub, _ptr(first)) != 0:
        raise ValueError("bad subband partition %d / %d" % (nchan, nsub))
    return first


def subband_freqs(nchan, f_lo, f_hi, nsub, mode):
    """Representative frequency F_s of every subband (Sec. 2.3)."""
    first = subband_first(nchan, nsub)
    F = np.array([lib().oracle_subband_freq(nchan, f_lo, f_hi, int(first[s]), int(first[s + 1]), mode)
                  for s in range(nsub)])
    if np.any(F <= 0):
        raise ValueError("bad subband frequency mode %r" % (mode,))
    return F


def subband_tables(nchan, f_lo, f_hi, tsamp, dms, n0, nsub, mode):
    """Tables of two-stage subband dedispersion (Sec. 2.3): the partition,
    F_s, the coarse DMs dm[j*N0] and their delays (Eq. coarse_delay), the
    residual shifts R [ndm][nsub] (Eq. residual)."""
    dms = np.ascontiguousarray(dms, dtype=np.float64)
    ndm = dms.size
    R = np.empty((ndm, nsub), dtype=np.int32)
    rc = lib().oracle_subband_residuals(nchan, f_lo, f_hi, tsamp, _ptr(dms), ndm, n0, nsub, mode, _ptr(R))
    if rc != 0:
        raise ValueError("oracle_subband_residuals failed (%d)" % rc)
    coarse = dms[::n0].copy()
    return dict(first=subband_first(nchan, nsub), F=subband_freqs(nchan, f_lo, f_hi, nsub, mode),
                coarse_dms=coarse, Dc=delay_table(nchan, f_lo, f_hi, tsamp, coarse), R=R, n0=int(n0),
                nsub=int(nsub), ndm=int(ndm), nchan=int(nchan))


def subband_effective_delays(tab):
    """Per-channel delay that the two stages apply for fine DM m:
    Deff[m][c] = D[j(m)][c] + R[m][s(c)] (stage 2 of Eq. stage2 inserted into
    Eq. stage1).  Reading: the plane of the two stages is the brute-force sum
    with this table, and nout = nsamp - max(Deff)."""
    first, Dc, R, n0 = tab["first"], tab["Dc"], tab["R"], tab["n0"]
    ndm, nchan = tab["ndm"], tab["nchan"]
    sub_of = np.repeat(np.arange(tab["nsub"]), np.diff(first))
    j = np.arange(ndm) // n0
    return (Dc[j, :].astype(np.int64) + R[:, sub_of].astype(np.int64)).astype(np.int32)


def subband_dedisperse(X, tab, nout=None):
    """Two-stage subband plane, Eqs. (stage1), (stage2) (Sec. 2.3), int32."""
    X = np.ascontiguousarray(X, dtype=np.uint8)
    nchan, nsamp = X.shape
    if nchan != tab["nchan"]:
        raise ValueError("table / data channel mismatch")
    if nout is None:
        nout = nsamp - int(subband_effective_delays(tab).max())
    if nout <= 0:
        raise ValueError("nout out of range")
    ndm = tab["ndm"]
    Y = np.empty((ndm, nout), dtype=np.int32)
    Dc = np.ascontiguousarray(tab["Dc"], dtype=np.int32)
    R = np.ascontiguousarray(tab["R"], dtype=np.int32)
    first = np.ascontiguousarray(tab["first"], dtype=np.int32)
    rc = lib().oracle_subband_dedisperse(_ptr(X), nchan, nsamp, _ptr(Dc), Dc.shape[0], _ptr(first), tab["nsub"],
                                         _ptr(R), ndm, tab["n0"], nout, _ptr(Y))
    if rc != 0:
        raise ValueError("oracle_subband_dedisperse failed (%d)" % rc)
    return Y


def downsample_sqlaw(X, D, vmax=255):
    """Square-law downsampling by D (Sec. 2.2), uint8 [nchan][ceil(nsamp/D)]."""
    X = np.ascontiguousarray(X, dtype=np.uint8)
    nchan, nsamp = X.shape
    out = np.empty((nchan, (nsamp + D - 1) // D), dtype=np.uint8)
    if lib().oracle_downsample_sqlaw(_ptr(X), nchan, nsamp, int(D), int(vmax), _ptr(out)) != 0:
        raise ValueError("oracle_downsample_sqlaw: bad arguments")
    return out


MAD_TO_SIGMA = 1.482602218505602   # sigma / MAD for a normal distribution


def zerodm(X):
    """Zero-DM filter (reading: channel mean rounded half up, re-centred at 128, clipped)."""
    X = np.ascontiguousarray(X, dtype=np.uint8)
    out = np.empty_like(X)
    if lib().oracle_zerodm(_ptr(X), X.shape[0], X.shape[1], _ptr(out)) != 0:
        raise ValueError("oracle_zerodm: bad arguments")
    return out


def row_robust(Y):
    """(median, MAD) of every plane row: lower medians, int64."""
    Y = np.ascontiguousarray(Y, dtype=np.int32)
    ndm, nout = Y.shape
    med = np.empty(ndm, dtype=np.int64)
    mad = np.empty(ndm, dtype=np.int64)
    lib().oracle_row_robust(_ptr(Y), ndm, nout, _ptr(med), _ptr(mad))
    return med, mad


def boxcar_snr_norm(Y, widths, mu, sigma):
    """Boxcar S/N with explicit per-row location and scale."""
    Y = np.ascontiguousarray(Y, dtype=np.int32)
    widths = np.ascontiguousarray(widths, dtype=np.int32)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    ndm, nout = Y.shape
    snr = np.empty((ndm, nout), dtype=np.float64)
    bw = np.empty((ndm, nout), dtype=np.int32)
    lib().oracle_boxcar_snr_norm(_ptr(Y), ndm, nout, _ptr(widths), widths.size, _ptr(mu), _ptr(sigma), _ptr(snr),
                                 _ptr(bw))
    return snr, bw


def boxcar_snr_robust(Y, widths):
    """Robust S/N: location = median, scale = 1.4826 * MAD of each row."""
    med, mad = row_robust(Y)
    return boxcar_snr_norm(Y, widths, med.astype(np.float64), MAD_TO_SIGMA * mad.astype(np.float64))


def threads():
    """Threads of the oracle's OpenMP team (what its parallel loops use)."""
    return int(lib().oracle_threads())
