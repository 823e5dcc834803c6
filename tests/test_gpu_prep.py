"""Parity of the preprocessing and normalisation kernels with the CPU oracle,
through the C ABI: square-law downsampling and the zero-DM filter (bit-exact),
channel-range plans for the multi-band search (tables identical, planes
bit-exact, F = L + H), median/MAD row statistics (exact) and the robust S/N
(|gpu - oracle| <= 1e-5 * max(|oracle|, 1))."""
import numpy as np
import pytest

import oracle
from conftest import C1, dm_list
from paper_2511_02328_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _lib():
    from paper_2511_02328_gb300 import _lib
    return _lib


# D <= 16384 takes the kernel's 32-bit arithmetic, larger D the 64-bit one
@pytest.mark.parametrize("shape,D", [((3, 1000), 1), ((5, 1001), 3), ((64, 4096), 8), ((7, 100003), 64),
                                     ((2, 40000), 16384), ((2, 70000), 32768), ((1, 17), 16), ((4096, 1 << 14), 4)])
def test_downsample_bit_exact(shape, D):
    rng = np.random.default_rng(shape[0] * 7 + D)
    X = rng.integers(0, 256, size=shape, dtype=np.uint8)
    X[0, :min(shape[1], 50)] = 255          # saturating bins
    X[-1, :min(shape[1], D)] = 255          # a whole bin at 255: the largest sums
    ref = oracle.downsample_sqlaw(X, D)
    x = torch.from_numpy(X).cuda()
    out = torch.empty(ref.shape, dtype=torch.uint8, device="cuda")
    _lib().af_downsample(x.data_ptr(), shape[0], shape[1], D, out.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)


def test_downsample_argument_errors():
    L = _lib()
    x = torch.zeros((2, 10), dtype=torch.uint8, device="cuda")
    for D in (0, 32769):
        with pytest.raises(L.AFError):
            L.af_downsample(x.data_ptr(), 2, 10, D, x.data_ptr())


# the 512-sample tile path (nsamp % 512 == 0, 16-byte aligned rows, at least 16 channels) and the generic kernel
@pytest.mark.parametrize("shape", [(1, 7), (2, 9), (31, 32), (1, 128), (5, 256), (64, 4096), (37, 10001),
                                   (4096, 8192), (4097, 96), (6144, 64), (255, 1 << 12), (8192, 1024),
                                   (16, 1 << 16), (1025, 1 << 15)])
@pytest.mark.parametrize("inplace", [False, True])
def test_zerodm_bit_exact(shape, inplace):
    rfi = synth.RFI(bursts=[(shape[1] // 3, 5, 60.0)], narrow_channels=[0])
    X = synth.filterbank(shape[0], shape[1], seed=shape[0] + shape[1], rfi=rfi)
    ref = oracle.zerodm(X)
    x = torch.from_numpy(X).cuda()
    out = x if inplace else torch.empty_like(x)
    _lib().af_zerodm(x.data_ptr(), shape[0], shape[1], out.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)


def test_channel_range_plans_multiband():
    # F = [0, nchan), L = lower half, H = upper half of the 256-channel band:
    # tables are the whole band's columns, planes are bit-exact, and F = L + H.
    from paper_2511_02328_gb300.search import Plan
    cfg = C1
    nchan, dms = cfg["nchan"], dm_list(cfg)
    D = oracle.delay_table(nchan, cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms)
    X = synth.filterbank(nchan, cfg["nsamp"], seed=21)
    x = torch.from_numpy(X).cuda()
    planes = {}
    for name, (c0, c1) in {"F": (0, nchan), "L": (0, nchan // 2), "H": (nchan // 2, nchan)}.items():
        p = Plan(nchan, cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms, channels=(c0, c1))
        assert np.array_equal(p.delays(), D[:, c0:c1])
        Y = p.dedisperse(x[c0:c1]).cpu().numpy()
        assert np.array_equal(Y, oracle.dedisperse(X[c0:c1], D[:, c0:c1]))
        planes[name] = Y
        p.close()
    n = planes["F"].shape[1]
    assert planes["H"].shape[1] > n and planes["L"].shape[1] == n
    assert np.array_equal(planes["F"], planes["L"][:, :n] + planes["H"][:, :n])


def test_band_limited_pulse_is_stronger_in_its_half():
    # A pulse only in the upper half of the band (Sec. 2.2: separate subbands
    # improve the visibility of band-limited signals): the H search reports a
    # higher S/N than the full-band search, at the same DM and TOA; the union of
    # the F, L, H candidates clusters to one event.
    from paper_2511_02328_gb300.search import Plan
    L = _lib()
    cfg = C1
    nchan, dms = cfg["nchan"], dm_list(cfg)
    offs = oracle.injection_offsets(nchan, cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], 250.0, 12000)
    amp = np.zeros(nchan, dtype=np.float32)
    amp[nchan // 2:] = synth.pulse_amplitude(14.0, nchan // 2, 8)
    X = synth.filterbank(nchan, cfg["nsamp"], seed=22, pulses=[synth.Pulse(offs, 8, amp)])
    best, allc = {}, []
    for name, (c0, c1) in {"F": (0, nchan), "L": (0, nchan // 2), "H": (nchan // 2, nchan)}.items():
        p = Plan(nchan, cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms, channels=(c0, c1))
        L.af_search_reserve(p.handle, cfg["nsamp"], 4096)
        c, n = L.af_search(p.handle, np.ascontiguousarray(X[c0:c1]), cfg["nsamp"], cfg["widths"], 7.0, 4096)
        near = c[(np.abs(dms[c["dm_idx"]] - 250.0) < 20) & (np.abs(c["abs_sample"] - 12000) < 50)]
        best[name] = float(near["snr"].max()) if near.size else 0.0
        allc.append(c)
        if name == "F":
            pf = p
        else:
            p.close()
    assert best["H"] > best["F"] > 7.0
    assert best["L"] < 7.0
    merged = L.af_cluster(pf.handle, np.concatenate(allc))
    ev = merged[(np.abs(dms[merged["dm_idx"]] - 250.0) < 20) & (np.abs(merged["abs_sample"] - 12000) < 50)]
    assert ev.size == 1 and abs(float(ev["snr"][0]) - best["H"]) < 1e-6
    pf.close()


def _robust_plane(seed, ndm, nout):
    rng = np.random.default_rng(seed)
    Y = rng.normal(300000, 700, size=(ndm, nout)).round().astype(np.int32)
    Y[1, ::37] += 90000                         # outliers
    Y[2, :] = 123456                            # constant row (MAD 0)
    if nout > 5:
        Y[3, :5] = [0, 10 ** 6, 3, 3, 3]        # wide range
    Y[4, :] = np.where(np.arange(nout) % 2 == 0, 0, 10 ** 6)      # two values: median at the mean - sigma bound
    Y[5, 0] = 2 * 10 ** 9                       # the first value (the kernel's pivot) an outlier
    Y[6, :] = rng.choice(np.array([-2 ** 31, 2 ** 31 - 1]), nout)  # the whole int32 range
    Y[7, :] = rng.exponential(1000.0, nout).round().astype(np.int32)  # skewed
    return Y


@pytest.mark.parametrize("nout", [1, 2, 3, 1000, 20001, 215261])
def test_robust_rowstats_exact(nout):
    """Median and MAD exact on noise, outliers, a constant row, two-valued and
    full-int32-range rows, an outlier first value and a skewed row."""
    Y = _robust_plane(nout, 8, nout)
    med, mad = oracle.row_robust(Y)
    L = _lib()
    p = L.af_plan(16, 1000.0, 1500.0, 1e-4, np.zeros(8))
    y = torch.from_numpy(Y).cuda()
    r = torch.empty((8, 2), dtype=torch.int64, device="cuda")
    L.af_rowstats_robust(p, y.data_ptr(), nout, r.data_ptr())
    torch.cuda.synchronize()
    got = r.cpu().numpy()
    assert np.array_equal(got[:, 0], med) and np.array_equal(got[:, 1], mad)
    L.af_plan_destroy(p)


def test_robust_snr_on_a_search_plane():
    from paper_2511_02328_gb300.search import Plan
    L = _lib()
    cfg = C1
    dms = dm_list(cfg)[:120]
    offs = oracle.injection_offsets(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], 60.0, 7000)
    rfi = synth.RFI(bursts=[(3000, 4, 50.0), (15000, 2, 90.0)])
    X = synth.filterbank(cfg["nchan"], cfg["nsamp"], seed=5, rfi=rfi,
                         pulses=[synth.Pulse(offs, 10, synth.pulse_amplitude(15.0, cfg["nchan"], 10))])
    p = Plan(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms)
    x = torch.from_numpy(X).cuda()
    Y = p.dedisperse(x)
    nout = Y.shape[1]
    snr = torch.empty(Y.shape, dtype=torch.float32, device="cuda")
    bw = torch.empty(Y.shape, dtype=torch.uint8, device="cuda")
    L.af_boxcar_snr_robust(p.handle, Y.data_ptr(), nout, 0, cfg["widths"], snr.data_ptr(), bw.data_ptr())
    torch.cuda.synchronize()
    ref, rbw = oracle.boxcar_snr_robust(Y.cpu().numpy(), cfg["widths"])
    got = snr.cpu().numpy().astype(np.float64)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    err = np.abs(got[fin] - ref[fin]) / np.maximum(1.0, np.abs(ref[fin]))
    assert float(err.max()) <= TOL
    agree = (bw.cpu().numpy().astype(np.int32) == np.where(rbw < 0, 255, rbw))
    assert agree.mean() > 0.999
    p.close()
