"""ctypes binding of libafgb.so (include/afgb.h), argument marshalling only.

Every function here has the name of the C entry point it wraps, takes plain
integers (device pointers as ints, e.g. tensor.data_ptr()) or numpy arrays
for host buffers, raises AFError on a non-zero status and returns the
outputs.  No computation happens in Python.  Importing this module on a
machine without the built library raises at once: there is no fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libafgb.so")

AF_OK, AF_EINVAL, AF_ENOMEM, AF_ENOBUFS, AF_ECUDA, AF_ETIMEOUT, AF_EOVERFLOW, AF_EAGAIN = range(8)
AF_MAX_WIDTHS = 32
AF_NO_WIDTH = 0xFF
AF_NOALLOC_MAX_ROWS = 4096
_NAMES = {0: "AF_OK", 1: "AF_EINVAL", 2: "AF_ENOMEM", 3: "AF_ENOBUFS", 4: "AF_ECUDA", 5: "AF_ETIMEOUT",
          6: "AF_EOVERFLOW", 7: "AF_EAGAIN"}


class AFError(RuntimeError):
    def __init__(self, code, fn, msg):
        super().__init__("%s failed: %s: %s" % (fn, _NAMES.get(code, code), msg))
        self.code = code


class RowStats(ctypes.Structure):
    _fields_ = [("sum", ctypes.c_int64), ("sumsq", ctypes.c_int64)]


class Cand(ctypes.Structure):
    _fields_ = [("dm_idx", ctypes.c_int32), ("t", ctypes.c_int32), ("width", ctypes.c_int32),
                ("snr", ctypes.c_float), ("abs_sample", ctypes.c_int64)]


CAND_DTYPE = np.dtype([("dm_idx", np.int32), ("t", np.int32), ("width", np.int32), ("snr", np.float32),
                       ("abs_sample", np.int64)])
assert CAND_DTYPE.itemsize == ctypes.sizeof(Cand) == 24

_P = ctypes.c_void_p
_I = ctypes.c_int
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double
_F = ctypes.c_float

# name -> argtypes (all return int unless listed in _RESTYPE)
SIGNATURES = {
    "af_last_error": [],
    "af_version": [],
    "af_plan": [_P, _I, _D, _D, _D, _P, _I],
    "af_plan_subband": [_P, _I, _D, _D, _D, _P, _I, _I, _I, _I, _I64],
    "af_plan_subband_info": [_P, _P, _P, _P, _P, _P, _P, _P, _P],
    "af_plan_channels": [_P, _I, _D, _D, _D, _P, _I, _I, _I],
    "af_downsample": [_P, _I, _I64, _I, _P, _P],
    "af_zerodm": [_P, _I, _I64, _P, _P],
    "af_rowstats_robust": [_P, _P, _I64, _P, _P],
    "af_boxcar_snr_robust": [_P, _P, _I64, _P, _P, _I, _P, _P, _P],
    "af_grid": [_P, _I, _I64, _I64, _I, _P, _P, _P],
    "af_diag_int_rates": [_P, _P],
    "af_diag_smem_rate": [_P],
    "af_diag_bounded_wait": [_I, _I64, _P],
    "af_plan_destroy": [_P],
    "af_plan_delays": [_P, _P, _P],
    "af_plan_info": [_P, _P, _P, _P, _P],
    "af_plan_nout": [_P, _I64, _P],
    "af_plan_check": [_P],
    "af_plan_kernel": [_P, _P, _P, _P, _P],
    "af_dedisperse_reserve": [_P, _I64],
    "af_dedisperse_workspace_size": [_P, _I64, _P],
    "af_search_workspace_size": [_P, _I64, _I32, _P],
    "af_dedisperse_timing": [_P, _I],
    "af_search_timing": [_P, _I],
    "af_search_times": [_P, _P, _P, _P],
    "af_dedisperse_times": [_P, _I, _P, _P, _P, _P],
    "af_dedisperse": [_P, _P, _I64, _P, _P, _P],
    "af_rowstats": [_P, _P, _I64, _P, _P],
    "af_boxcar_snr": [_P, _P, _I64, _P, _P, _I, _P, _P, _P],
    "af_boxcar_snr_noalloc": [_P, _I, _I64, _I, _P, _I, _P, _P, _P],
    "af_candidates": [_P, _P, _P, _I64, _P, _I, _F, _I64, _P, _I32, _P, _P],
    "af_cluster": [_P, _P, _I32, _D, _D, _P, _P],
    "af_search_reserve": [_P, _I64, _I32],
    "af_search": [_P, _P, _I64, _P, _I, _F, _P, _I32, _P, _P],
    "af_batch_build": [_P, _P, _I, ctypes.c_size_t],
    "af_batch_run": [_P, _P],
    "af_batch_candidates": [_P, _I, _P, _I32, _P],
    "af_batch_buffers": [_P, _I, _P, _P, _P, _P],
    "af_batch_shape": [_P, _P, _P, _P, _P],
    "af_batch_tuning": [_P, _I, _P, _P, _P, _P],
    "af_batch_destroy": [_P],
    "af_stream_open": [_P, _P],
    "af_stream_push": [_P, _I, _P, _I64, _I64, _I64],
    "af_stream_poll": [_P, _P, _I],
    "af_stream_release": [_P, _I32],
    "af_stream_result_plane": [_P, _I32, _P, _P, _P],
    "af_stream_info": [_P, _P, _P, _P],
    "af_stream_stats": [_P, _P],
    "af_stream_snapshot": [_P, _I, _P, _P, _P],
    "af_stream_restore": [_P, _I, _P, _I64, _I64],
    "af_stream_close": [_P],
    "af_stream_classify": [_P, _I32, _P, _P, _I32, _P],
    "af_stream_cluster": [_P, _P, _I32, _P, _P],
    "af_nn_gemm": [_I, _I, _P, _I, _P, _I, _I, _I, _I, _I, _P, _I, _P, _P],
    "af_cutouts": [_P, _P, _I64, _P, _I64, _P, _I32, _P, _P],
    "af_model_create": [_P, _I, ctypes.c_uint64],
    "af_model_destroy": [_P],
    "af_model_nparams": [_P, _P],
    "af_model_set_params": [_P, _P, _I64],
    "af_model_get_params": [_P, _P, _I64],
    "af_model_get_grads": [_P, _P, _I64],
    "af_model_save": [_P, ctypes.c_char_p],
    "af_model_load": [_P, ctypes.c_char_p],
    "af_model_forward": [_P, _P, _I32, _P, _P, _P],
    "af_model_backward": [_P, _P, _P, _I32, _P, _P],
    "af_train_step": [_P, _P, _P, _I32, _F, _P, _P],
    "af_classify": [_P, _P, _P, _I64, _P, _I64, _P, _I32, _P, _P],
}
_RESTYPE = {"af_last_error": ctypes.c_char_p, "af_version": ctypes.c_char_p}

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libafgb.so is not built: run paper_2511_02328_gb300.build.build() "
                              "(or __graft_entry__.build()) first")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _RESTYPE.get(name, ctypes.c_int)
        _lib = L
    return _lib


def _check(rc, fn, allow=()):
    if rc != AF_OK and rc not in allow:
        raise AFError(rc, fn, lib().af_last_error().decode())
    return rc


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(_P)


def af_last_error():
    return lib().af_last_error().decode()


def af_version():
    return lib().af_version().decode()


def af_plan(nchan, f_lo, f_hi, tsamp, dm_list):
    dms, pd = _host(dm_list, np.float64)
    h = _P()
    _check(lib().af_plan(ctypes.byref(h), int(nchan), float(f_lo), float(f_hi), float(tsamp), pd, int(dms.size)),
           "af_plan")
    return h.value


def af_plan_channels(nchan, f_lo, f_hi, tsamp, dm_list, c0, c1):
    dms, pd = _host(dm_list, np.float64)
    h = _P()
    _check(lib().af_plan_channels(ctypes.byref(h), int(nchan), float(f_lo), float(f_hi), float(tsamp), pd,
                                  int(dms.size), int(c0), int(c1)), "af_plan_channels")
    return h.value


def af_downsample(d_in, nchan, nsamp, D, d_out, stream=0):
    _check(lib().af_downsample(d_in, int(nchan), int(nsamp), int(D), d_out, stream or None), "af_downsample")


def af_zerodm(d_in, nchan, nsamp, d_out, stream=0):
    _check(lib().af_zerodm(d_in, int(nchan), int(nsamp), d_out, stream or None), "af_zerodm")


def af_rowstats_robust(plan, d_plane, nout, d_robust, stream=0):
    _check(lib().af_rowstats_robust(plan, d_plane, int(nout), d_robust, stream or None), "af_rowstats_robust")


def af_boxcar_snr_robust(plan, d_plane, nout, d_robust, widths, d_best_snr, d_best_w=0, stream=0):
    w, pw = _host(widths, np.int32)
    _check(lib().af_boxcar_snr_robust(plan, d_plane, int(nout), d_robust or None, pw, int(w.size), d_best_snr,
                                      d_best_w or None, stream or None), "af_boxcar_snr_robust")


def af_grid(d_plane, ndm, nout, ns, M, d_out, d_work, stream=0):
    _check(lib().af_grid(d_plane, int(ndm), int(nout), int(ns), int(M), d_out, d_work, stream or None), "af_grid")


def af_diag_int_rates():
    """(int32 2-input adds per second, dedispersion-pattern sample adds per second)."""
    a, b = _D(), _D()
    _check(lib().af_diag_int_rates(ctypes.byref(a), ctypes.byref(b)), "af_diag_int_rates")
    return a.value, b.value


def af_diag_smem_rate():
    """Measured shared-memory load bandwidth of the current device (bytes/s)."""
    a = ctypes.c_double()
    _check(lib().af_diag_smem_rate(ctypes.byref(a)), "af_diag_smem_rate")
    return a.value


def af_diag_bounded_wait(arrive, polls):
    """Bounded-wait probe: (status, ms).  AF_ETIMEOUT when nothing arrived and
    the wait gave up after `polls` polls, AF_OK when the arrival came."""
    ms = ctypes.c_float()
    rc = _check(lib().af_diag_bounded_wait(int(arrive), int(polls), ctypes.byref(ms)), "af_diag_bounded_wait",
                allow=(AF_ETIMEOUT,))
    return rc, ms.value


AF_FS_MEDIAN = 0
AF_FS_INVSQ = 1


def af_plan_subband(nchan, f_lo, f_hi, tsamp, dm_list, n0, nsub, fs_mode=AF_FS_INVSQ, block_len=0):
    dms, pd = _host(dm_list, np.float64)
    h = _P()
    _check(lib().af_plan_subband(ctypes.byref(h), int(nchan), float(f_lo), float(f_hi), float(tsamp), pd,
                                 int(dms.size), int(n0), int(nsub), int(fs_mode), int(block_len)),
           "af_plan_subband")
    return h.value


def af_plan_subband_info(plan):
    """dict(n0, nsub, ncoarse, first, F, Dc, R, block_len) of a subband plan."""
    nchan, ndm, _, _ = af_plan_info(plan)
    n0, nsub, ncoarse, L = _I(), _I(), _I(), _I64()
    _check(lib().af_plan_subband_info(plan, ctypes.byref(n0), ctypes.byref(nsub), ctypes.byref(ncoarse), None,
                                      None, None, None, ctypes.byref(L)), "af_plan_subband_info")
    first = np.empty(nsub.value + 1, dtype=np.int32)
    F = np.empty(nsub.value, dtype=np.float64)
    Dc = np.empty((ncoarse.value, nchan), dtype=np.int32)
    R = np.empty((ndm, nsub.value), dtype=np.int32)
    _check(lib().af_plan_subband_info(plan, None, None, None, first.ctypes.data_as(_P), F.ctypes.data_as(_P),
                                      Dc.ctypes.data_as(_P), R.ctypes.data_as(_P), None), "af_plan_subband_info")
    return dict(n0=n0.value, nsub=nsub.value, ncoarse=ncoarse.value, first=first, F=F, Dc=Dc, R=R,
                block_len=L.value)


def af_plan_destroy(plan):
    _check(lib().af_plan_destroy(plan), "af_plan_destroy")


def af_plan_info(plan):
    nchan, ndm, dmax, tsamp = _I(), _I(), _I32(), _D()
    _check(lib().af_plan_info(plan, ctypes.byref(nchan), ctypes.byref(ndm), ctypes.byref(dmax),
                              ctypes.byref(tsamp)), "af_plan_info")
    return nchan.value, ndm.value, dmax.value, tsamp.value


PATH_SIMPLE, PATH_TILE, PATH_SUBBAND, PATH_PAIRS = 0, 1, 2, 3


def af_plan_kernel(plan):
    """(path, ring, spread, group) of the kernel that dedisperses this plan."""
    path, ring, spread, group = _I(), _I(), _I32(), _I()
    _check(lib().af_plan_kernel(plan, ctypes.byref(path), ctypes.byref(ring), ctypes.byref(spread),
                                ctypes.byref(group)), "af_plan_kernel")
    return path.value, ring.value, spread.value, group.value


def af_dedisperse_reserve(plan, max_nsamp):
    _check(lib().af_dedisperse_reserve(plan, max_nsamp), "af_dedisperse_reserve")


def af_dedisperse_workspace_size(plan, max_nsamp):
    b = ctypes.c_size_t()
    _check(lib().af_dedisperse_workspace_size(plan, max_nsamp, ctypes.byref(b)), "af_dedisperse_workspace_size")
    return b.value


def af_search_workspace_size(plan, max_nsamp, cap):
    b = ctypes.c_size_t()
    _check(lib().af_search_workspace_size(plan, max_nsamp, cap, ctypes.byref(b)), "af_search_workspace_size")
    return b.value


def af_search_timing(plan, enable):
    _check(lib().af_search_timing(plan, int(bool(enable))), "af_search_timing")


def af_search_times(plan):
    """(copy wait, dedispersion, S/N + candidates) of the last timed af_search call, ms."""
    a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    _check(lib().af_search_times(plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "af_search_times")
    return a.value, b.value, c.value


def af_dedisperse_timing(plan, ncalls):
    _check(lib().af_dedisperse_timing(plan, ncalls), "af_dedisperse_timing")


def af_dedisperse_times(plan, call):
    """(stage-1 ms, stage-2 ms, row-buffer bytes, row-window bytes copied) of timed call slot `call`."""
    r, t, b, c = ctypes.c_float(), ctypes.c_float(), _I64(), _I64()
    _check(lib().af_dedisperse_times(plan, call, ctypes.byref(r), ctypes.byref(t), ctypes.byref(b),
                                     ctypes.byref(c)), "af_dedisperse_times")
    return r.value, t.value, b.value, c.value


def af_plan_delays(plan):
    nchan, ndm, _, _ = af_plan_info(plan)
    out = np.empty((ndm, nchan), dtype=np.int32)
    dmax = _I32()
    _check(lib().af_plan_delays(plan, out.ctypes.data_as(_P), ctypes.byref(dmax)), "af_plan_delays")
    return out, dmax.value


def af_plan_check(plan):
    _check(lib().af_plan_check(plan), "af_plan_check")


def af_plan_nout(plan, nsamp):
    n = _I64()
    _check(lib().af_plan_nout(plan, int(nsamp), ctypes.byref(n)), "af_plan_nout")
    return n.value


def af_dedisperse(plan, d_in, nsamp, d_plane, d_stats=0, stream=0):
    _check(lib().af_dedisperse(plan, d_in, int(nsamp), d_plane, d_stats or None, stream or None), "af_dedisperse")


def af_rowstats(plan, d_plane, nout, d_stats, stream=0):
    _check(lib().af_rowstats(plan, d_plane, int(nout), d_stats, stream or None), "af_rowstats")


def af_boxcar_snr(plan, d_plane, nout, d_stats, widths, d_best_snr, d_best_w=0, stream=0):
    w, pw = _host(widths, np.int32)
    _check(lib().af_boxcar_snr(plan, d_plane, int(nout), d_stats or None, pw, int(w.size), d_best_snr,
                               d_best_w or None, stream or None), "af_boxcar_snr")


def af_boxcar_snr_noalloc(d_plane, ndm, nout, nchan, widths, d_best_snr, d_best_w=0, stream=0):
    w, pw = _host(widths, np.int32)
    _check(lib().af_boxcar_snr_noalloc(d_plane, int(ndm), int(nout), int(nchan), pw, int(w.size), d_best_snr,
                                       d_best_w or None, stream or None), "af_boxcar_snr_noalloc")


def af_candidates(plan, d_best_snr, d_best_w, nout, widths, thresh, sample0, d_out, cap, d_count, stream=0):
    w, pw = _host(widths, np.int32)
    _check(lib().af_candidates(plan, d_best_snr, d_best_w, int(nout), pw, int(w.size), float(thresh),
                               int(sample0), d_out or None, int(cap), d_count, stream or None), "af_candidates")


def af_cluster(plan, cands, dm_tol=20.0, toa_tol=0.2):
    """cands: numpy array of CAND_DTYPE (sorted in place by (dm_idx, t))."""
    c = np.ascontiguousarray(cands, dtype=CAND_DTYPE)
    out = np.empty_like(c)
    n = _I32()
    _check(lib().af_cluster(plan, c.ctypes.data_as(_P), int(c.size), float(dm_tol), float(toa_tol),
                            out.ctypes.data_as(_P), ctypes.byref(n)), "af_cluster")
    return out[: n.value]


def af_search_reserve(plan, max_nsamp, cap):
    _check(lib().af_search_reserve(plan, int(max_nsamp), int(cap)), "af_search_reserve")


def af_search(plan, h_in, nsamp, widths, thresh, cap, stream=0, out=None):
    """h_in: host pointer (int) or a C-contiguous uint8 numpy array [nchan][nsamp].
    Returns (candidates sorted by (dm_idx, t), total count)."""
    w, pw = _host(widths, np.int32)
    if isinstance(h_in, np.ndarray):
        keep = np.ascontiguousarray(h_in, dtype=np.uint8)
        ptr = keep.ctypes.data
    else:
        ptr = int(h_in)
    if out is None:
        out = np.empty(max(int(cap), 1), dtype=CAND_DTYPE)
    n = _I32()
    _check(lib().af_search(plan, ptr, int(nsamp), pw, int(w.size), float(thresh), out.ctypes.data_as(_P),
                           int(cap), ctypes.byref(n), stream or None), "af_search", allow=(AF_EOVERFLOW,))
    return out[: min(n.value, int(cap))], n.value


class BeamDesc(ctypes.Structure):
    _fields_ = [("nchan", ctypes.c_int), ("f_lo", ctypes.c_double), ("f_hi", ctypes.c_double),
                ("tsamp", ctypes.c_double), ("dm_list", ctypes.c_void_p), ("ndm", ctypes.c_int),
                ("d_in", ctypes.c_void_p), ("nsamp", ctypes.c_int64), ("widths", ctypes.c_void_p),
                ("nw", ctypes.c_int), ("thresh", ctypes.c_float), ("cap", ctypes.c_int32)]


def af_batch_build(beams, hbm_budget=0):
    """beams: list of dicts with keys nchan, f_lo, f_hi, tsamp, dm_list, d_in (device ptr),
    nsamp, widths, thresh, cap.  Returns the batch handle."""
    keep = []
    arr = (BeamDesc * len(beams))()
    for i, b in enumerate(beams):
        dms, pd = _host(b["dm_list"], np.float64)
        w, pw = _host(b["widths"], np.int32)
        keep += [dms, w]
        arr[i] = BeamDesc(int(b["nchan"]), float(b["f_lo"]), float(b["f_hi"]), float(b["tsamp"]), pd, int(dms.size),
                          int(b["d_in"]), int(b["nsamp"]), pw, int(w.size), float(b["thresh"]), int(b["cap"]))
    h = _P()
    _check(lib().af_batch_build(ctypes.byref(h), arr, len(beams), int(hbm_budget)), "af_batch_build")
    return h.value


def af_batch_run(batch, stream=0):
    _check(lib().af_batch_run(batch, stream or None), "af_batch_run")


def af_batch_candidates(batch, beam, cap):
    out = np.empty(max(int(cap), 1), dtype=CAND_DTYPE)
    n = _I32()
    _check(lib().af_batch_candidates(batch, int(beam), out.ctypes.data_as(_P), int(cap), ctypes.byref(n)),
           "af_batch_candidates", allow=(AF_EOVERFLOW,))
    return out[: min(n.value, int(cap))], n.value


def af_batch_buffers(batch, beam):
    pl, sn, bw, no = _P(), _P(), _P(), _I64()
    _check(lib().af_batch_buffers(batch, int(beam), ctypes.byref(pl), ctypes.byref(sn), ctypes.byref(bw),
                                  ctypes.byref(no)), "af_batch_buffers")
    return pl.value, sn.value, bw.value, no.value


def af_batch_shape(batch):
    nw, m, ms, fc = _I(), _I(), _F(), _I()
    _check(lib().af_batch_shape(batch, ctypes.byref(nw), ctypes.byref(m), ctypes.byref(ms), ctypes.byref(fc)),
           "af_batch_shape")
    return nw.value, m.value, ms.value, bool(fc.value)


def af_batch_tuning(batch):
    """Every candidate the autotuner timed: list of dict(kind, p1, p2, ms)."""
    out = []
    kind, p1, p2, ms = _I(), _I(), _I(), _F()
    for i in range(64):
        rc = lib().af_batch_tuning(batch, i, ctypes.byref(kind), ctypes.byref(p1), ctypes.byref(p2), ctypes.byref(ms))
        if rc != AF_OK:
            break
        out.append(dict(kind=kind.value, p1=p1.value, p2=p2.value, ms=ms.value))
    return out


def af_batch_destroy(batch):
    _check(lib().af_batch_destroy(batch), "af_batch_destroy")


class StreamCfg(ctypes.Structure):
    _fields_ = [("nbeams", _I), ("nchan", _I), ("f_lo", _D), ("f_hi", _D), ("tsamp", _D), ("dm_list", _P),
                ("ndm", _I), ("window", _I64), ("widths", _P), ("nw", _I), ("thresh", _F), ("cap", _I32),
                ("hbm_budget", ctypes.c_size_t), ("max_slots", _I), ("timeout_ms", _I)]


class StreamResult(ctypes.Structure):
    _fields_ = [("beam", _I), ("seq", _I64), ("sample0", _I64), ("slot", _I32), ("count", _I32), ("total", _I32),
                ("cands", _P), ("latency_ms", _D), ("status", _I)]


class StreamStats(ctypes.Structure):
    _fields_ = [("windows", _I64), ("launches", _I64), ("max_inflight", _I), ("slots", _I), ("p50_ms", _D),
                ("p99_ms", _D), ("max_ms", _D), ("wall_s", _D), ("work", _D), ("rate", _D)]


def af_stream_open(nbeams, nchan, f_lo, f_hi, tsamp, dm_list, window, widths, thresh, cap, hbm_budget=0,
                   max_slots=0, timeout_ms=60000):
    dms, pd = _host(dm_list, np.float64)
    w, pw = _host(widths, np.int32)
    cfg = StreamCfg(int(nbeams), int(nchan), float(f_lo), float(f_hi), float(tsamp), pd, int(dms.size), int(window),
                    pw, int(w.size), float(thresh), int(cap), int(hbm_budget), int(max_slots), int(timeout_ms))
    h = _P()
    _check(lib().af_stream_open(ctypes.byref(h), ctypes.byref(cfg)), "af_stream_open")
    return h.value


def af_stream_push(stream, beam, h_data, seq):
    """h_data: uint8 [nchan][nsamp] numpy array whose rows are contiguous (a
    column slice of a larger C-contiguous array is passed with its pitch),
    or a tuple (ptr, nsamp, pitch)."""
    if isinstance(h_data, np.ndarray):
        a = h_data
        if a.dtype != np.uint8 or a.ndim != 2 or a.strides[1] != 1:
            a = np.ascontiguousarray(a, dtype=np.uint8)
        ptr, nsamp, pitch = a.ctypes.data, a.shape[1], a.strides[0]
    else:
        ptr, nsamp, pitch = h_data
    return _check(lib().af_stream_push(stream, int(beam), ptr, int(nsamp), int(pitch), int(seq)), "af_stream_push")


def af_stream_poll(stream, timeout_ms=60000):
    """Returns a dict (beam, seq, sample0, slot, cands, total, latency_ms, status) or None."""
    r = StreamResult()
    rc = lib().af_stream_poll(stream, ctypes.byref(r), int(timeout_ms))
    if rc == AF_EAGAIN:
        return None
    _check(rc, "af_stream_poll")
    cands = np.empty(0, dtype=CAND_DTYPE)
    if r.count > 0:
        buf = (ctypes.c_char * (r.count * CAND_DTYPE.itemsize)).from_address(r.cands)
        cands = np.frombuffer(buf, dtype=CAND_DTYPE).copy()
    return dict(beam=r.beam, seq=r.seq, sample0=r.sample0, slot=r.slot, cands=cands, total=r.total,
                latency_ms=r.latency_ms, status=r.status)


def af_stream_release(stream, slot):
    _check(lib().af_stream_release(stream, int(slot)), "af_stream_release")


def af_stream_result_plane(stream, slot):
    pl, sn, no = _P(), _P(), _I64()
    _check(lib().af_stream_result_plane(stream, int(slot), ctypes.byref(pl), ctypes.byref(sn), ctypes.byref(no)),
           "af_stream_result_plane")
    return pl.value, sn.value, no.value


def af_stream_info(stream):
    hop, dmax, ns = _I64(), _I64(), _I()
    _check(lib().af_stream_info(stream, ctypes.byref(hop), ctypes.byref(dmax), ctypes.byref(ns)), "af_stream_info")
    return hop.value, dmax.value, ns.value


def af_stream_stats(stream):
    st = StreamStats()
    _check(lib().af_stream_stats(stream, ctypes.byref(st)), "af_stream_stats")
    return {k: getattr(st, k) for k, _ in StreamStats._fields_}


def af_stream_snapshot(stream, beam, nchan, dmax):
    ov = np.empty((nchan, max(dmax, 0)), dtype=np.uint8)
    ns, nx = _I64(), _I64()
    _check(lib().af_stream_snapshot(stream, int(beam), ov.ctypes.data_as(_P), ctypes.byref(ns), ctypes.byref(nx)),
           "af_stream_snapshot")
    return ov, ns.value, nx.value


def af_stream_restore(stream, beam, overlap, next_seq, next_sample):
    ov = np.ascontiguousarray(overlap, dtype=np.uint8)
    _check(lib().af_stream_restore(stream, int(beam), ov.ctypes.data_as(_P), int(next_seq), int(next_sample)),
           "af_stream_restore")


def af_stream_classify(stream, slot, model, cands):
    """cands: CAND_DTYPE array (host).  Returns P(pulse) per candidate."""
    c = np.ascontiguousarray(cands, dtype=CAND_DTYPE)
    prob = np.empty(max(c.size, 1), dtype=np.float32)
    _check(lib().af_stream_classify(stream, int(slot), model, c.ctypes.data_as(_P), int(c.size),
                                    prob.ctypes.data_as(_P)), "af_stream_classify")
    return prob[: c.size]


def af_stream_cluster(stream, cands):
    c = np.ascontiguousarray(cands, dtype=CAND_DTYPE).copy()
    out = np.empty(max(c.size, 1), dtype=CAND_DTYPE)
    n = _I32()
    _check(lib().af_stream_cluster(stream, c.ctypes.data_as(_P), int(c.size), out.ctypes.data_as(_P),
                                   ctypes.byref(n)), "af_stream_cluster")
    return out[: n.value]


def af_stream_close(stream):
    _check(lib().af_stream_close(stream), "af_stream_close")


NPARAMS = 23570


def af_nn_gemm(layout, epi, d_a, lda, d_b, ldb, M, N, K, splits, d_c, ldc, d_bias=0, stream=0):
    _check(lib().af_nn_gemm(int(layout), int(epi), d_a, int(lda), d_b, int(ldb), int(M), int(N), int(K), int(splits),
                            d_c, int(ldc), d_bias or None, stream or None), "af_nn_gemm")


def af_cutouts(plan, d_in, nsamp, d_plane, nout, d_cands, n, d_out, stream=0):
    _check(lib().af_cutouts(plan, d_in, int(nsamp), d_plane, int(nout), d_cands or None, int(n), d_out or None,
                            stream or None), "af_cutouts")


def af_model_create(max_batch, seed=0):
    h = _P()
    _check(lib().af_model_create(ctypes.byref(h), int(max_batch), int(seed)), "af_model_create")
    return h.value


def af_model_destroy(model):
    _check(lib().af_model_destroy(model), "af_model_destroy")


def af_model_nparams(model):
    n = _I64()
    _check(lib().af_model_nparams(model, ctypes.byref(n)), "af_model_nparams")
    return n.value


def af_model_set_params(model, params):
    p, pp = _host(params, np.float32)
    _check(lib().af_model_set_params(model, pp, int(p.size)), "af_model_set_params")


def af_model_get_params(model):
    out = np.empty(af_model_nparams(model), dtype=np.float32)
    _check(lib().af_model_get_params(model, out.ctypes.data_as(_P), int(out.size)), "af_model_get_params")
    return out


def af_model_get_grads(model):
    out = np.empty(af_model_nparams(model), dtype=np.float32)
    _check(lib().af_model_get_grads(model, out.ctypes.data_as(_P), int(out.size)), "af_model_get_grads")
    return out


def af_model_save(model, path):
    _check(lib().af_model_save(model, str(path).encode()), "af_model_save")


def af_model_load(model, path):
    _check(lib().af_model_load(model, str(path).encode()), "af_model_load")


def af_model_forward(model, d_x, n, d_logits=0, d_prob=0, stream=0):
    _check(lib().af_model_forward(model, d_x, int(n), d_logits or None, d_prob or None, stream or None),
           "af_model_forward")


def af_model_backward(model, d_x, d_y, n, d_loss=0, stream=0):
    _check(lib().af_model_backward(model, d_x, d_y, int(n), d_loss or None, stream or None), "af_model_backward")


def af_train_step(model, d_x, d_y, n, lr, d_loss=0, stream=0):
    _check(lib().af_train_step(model, d_x, d_y, int(n), float(lr), d_loss or None, stream or None), "af_train_step")


def af_classify(model, plan, d_in, nsamp, d_plane, nout, d_cands, n, d_prob, stream=0):
    _check(lib().af_classify(model, plan, d_in, int(nsamp), d_plane, int(nout), d_cands or None, int(n), d_prob,
                             stream or None), "af_classify")
