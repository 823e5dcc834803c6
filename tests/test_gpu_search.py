"""Parity of the CUDA search path with the CPU oracle, through the C ABI.

Plane: bit-exact.  S/N: |gpu - oracle| <= 1e-5 * max(|oracle|, 1) (float32
kernel vs fp64 oracle).  Best width and candidates: identical wherever the
decision is not within that tolerance of a tie or of the threshold."""
import numpy as np
import pytest

import oracle
from conftest import C1, C2, dm_list
from paper_2511_02328_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _plan(cfg, dms=None):
    from paper_2511_02328_gb300.search import Plan
    dms = dm_list(cfg) if dms is None else dms
    return Plan(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms)


def _snr_close(got, ref):
    got = got.astype(np.float64)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    err = np.abs(got[fin] - ref[fin]) / np.maximum(1.0, np.abs(ref[fin]))
    assert err.size == 0 or float(err.max()) <= TOL, float(err.max())


def _widths_agree(bw_got, bw_ref, plane, widths):
    """Best-width indices must agree except where the two best widths' S/N
    are within tolerance of each other (an fp tie)."""
    bad = np.argwhere(bw_got.astype(np.int32) != np.where(bw_ref < 0, 255, bw_ref))
    if bad.size == 0:
        return
    # recompute the contested entries in the oracle at both widths
    for d, t in bad[:200]:
        row = plane[d:d + 1]
        s, _ = oracle.boxcar_snr(row, [widths[int(bw_ref[d, t])]])
        s2, _ = oracle.boxcar_snr(row, [widths[int(bw_got[d, t])]])
        assert abs(s[0, t] - s2[0, t]) <= 2 * TOL * max(1.0, abs(s[0, t])), (d, t)


def _cands_agree(got, ref, ref_snr, thresh):
    """Returns the number of (d, t) on which the lists differ, every one of
    them checked to be an fp tie."""
    g = {(int(c["dm_idx"]), int(c["t"])) for c in got}
    r = {(c[0], c[1]) for c in ref}
    for (d, t) in g ^ r:
        # a difference is only allowed where the decision is an fp tie:
        # S/N at the threshold, or equal to a neighbour within tolerance
        s = ref_snr[d, t]
        near_thr = abs(s - thresh) <= TOL * max(1.0, abs(s))
        lo, hi = max(0, t - 300), min(ref_snr.shape[1], t + 301)
        near_tie = np.any((np.abs(ref_snr[d, lo:hi] - s) <= 2 * TOL * max(1.0, abs(s))) & (np.arange(lo, hi) != t))
        assert near_thr or near_tie, (d, t, s)
    return len(g ^ r)


def test_delay_table_identical():
    for cfg in (C1, C2):
        p = _plan(cfg)
        D = oracle.delay_table(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dm_list(cfg))
        assert np.array_equal(p.delays(), D)
        assert p.dmax == int(D.max())
        p.close()


@pytest.fixture(scope="module")
def c1_data():
    cfg = C1
    offs = oracle.injection_offsets(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], 300.0, 8000)
    x = synth.filterbank(cfg["nchan"], cfg["nsamp"], seed=1,
                         pulses=[synth.Pulse(offs, 10, synth.pulse_amplitude(15.0, cfg["nchan"], 10))])
    D = oracle.delay_table(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dm_list(cfg))
    Y = oracle.dedisperse(x, D)
    snr, bw = oracle.boxcar_snr(Y, cfg["widths"])
    return x, D, Y, snr, bw


def test_c1_full_parity(c1_data):
    x, D, Y, ref_snr, ref_bw = c1_data
    cfg = C1
    p = _plan(cfg)
    xd = torch.from_numpy(x).cuda()
    stats = torch.empty((p.ndm, 2), dtype=torch.int64, device="cuda")
    plane = p.dedisperse(xd, stats=stats)
    snr, bw = p.boxcar_snr(plane, cfg["widths"], stats=stats)
    out, cnt = p.candidates(snr, bw, cfg["widths"], 8.0)
    torch.cuda.synchronize()
    assert np.array_equal(plane.cpu().numpy(), Y)
    S, Q = oracle.rowstats(Y)
    st = stats.cpu().numpy()
    assert np.array_equal(st[:, 0], S) and np.array_equal(st[:, 1], Q)
    _snr_close(snr.cpu().numpy(), ref_snr)
    _widths_agree(bw.cpu().numpy(), ref_bw, Y, cfg["widths"])
    got, n = p.cands_to_numpy(out, cnt)
    ref, nref = oracle.peaks(ref_snr, ref_bw, cfg["widths"], 8.0)
    ndiff = _cands_agree(got, ref, ref_snr, 8.0)
    assert len(got) == n and abs(n - nref) <= ndiff
    # the injected pulse is the strongest candidate, at DM 300
    best = got[np.argmax(got["snr"])]
    assert int(best["dm_idx"]) == 300
    p.close()


def test_stats_computed_internally(c1_data):
    x, D, Y, ref_snr, _ = c1_data
    p = _plan(C1)
    plane = p.dedisperse(torch.from_numpy(x).cuda())
    snr, _ = p.boxcar_snr(plane, C1["widths"])           # d_stats = NULL -> plan scratch
    torch.cuda.synchronize()
    _snr_close(snr.cpu().numpy(), ref_snr)
    p.close()


def test_host_search_equals_device_path(c1_data):
    x, D, Y, ref_snr, ref_bw = c1_data
    p = _plan(C1)
    cands, n = p.search_host(x, C1["widths"], 8.0, cap=1 << 16)
    ref, nref = oracle.peaks(ref_snr, ref_bw, C1["widths"], 8.0)
    _cands_agree(cands, ref, ref_snr, 8.0)
    assert len(cands) == n
    # keys sorted by (dm_idx, t)
    k = list(zip(cands["dm_idx"].tolist(), cands["t"].tolist()))
    assert k == sorted(k)
    # clustering keeps one cluster for the single injected pulse
    kept = p.cluster(cands)
    assert len(kept) >= 1 and int(kept[0]["dm_idx"]) == 300
    p.close()


def test_host_search_long_candidate_lists(c1_data):
    """Candidate lists shorter and longer than the 4096 af_search returns with
    its count (one copy back, or a second copy), and a capacity below both."""
    x, D, Y, ref_snr, ref_bw = c1_data
    p = _plan(C1)
    full = {}
    for thresh, cap in ((4.0, 1 << 16), (3.5, 1 << 16), (3.5, 5000)):
        cands, n = p.search_host(x, C1["widths"], thresh, cap=cap)
        ref, nref = oracle.peaks(ref_snr, ref_bw, C1["widths"], thresh)
        assert len(cands) == min(n, cap)
        if cap >= n:
            # the counts differ by no more than the fp ties the lists differ on
            assert abs(n - nref) <= _cands_agree(cands, ref, ref_snr, thresh)
            full[thresh] = cands
        else:
            # a capacity below the total still reports the total; the `cap`
            # candidates returned (whichever the kernel appended first) are
            # entries of the whole list
            assert n == len(full[thresh])
            whole = {(int(c["dm_idx"]), int(c["t"])): c for c in full[thresh]}
            assert all(whole[(int(c["dm_idx"]), int(c["t"]))] == c for c in cands)
        k = list(zip(cands["dm_idx"].tolist(), cands["t"].tolist()))
        assert k == sorted(k)
    p.close()


SHAPES = [
    # nchan, f_lo, f_hi, tsamp, nsamp, dms
    (1, 1400.0, 1500.0, 1e-3, 100, [0.0]),
    (3, 1000.0, 1500.0, 1e-3, 257, [0.0, 7.0, 13.5]),
    (17, 1500.0, 1000.0, 5e-4, 1000, [30.0, 0.0, 12.0, 29.0, 5.5]),     # descending band, non-monotone DMs
    (65, 1000.0, 1500.0, 2e-4, 3001, list(np.arange(0, 40, 0.75))),
    (255, 1100.0, 1400.0, 1e-4, 5003, list(np.arange(0, 61, 1.0))),
    (300, 1000.0, 1500.0, 1e-4, 20011, [100.0]),                           # ndm = 1
    (129, 1200.0, 1300.0, 5e-5, 70001, list(np.arange(0, 200, 3.0))),
]


@pytest.mark.parametrize("kernel", ["auto", "pairs", "triples", "quads", "tile"])
@pytest.mark.parametrize("shape", SHAPES, ids=[str(i) for i in range(len(SHAPES))])
def test_random_shapes_bit_exact(shape, kernel, monkeypatch):
    """Every single-plan path (the default choice; rows of channel pairs or of
    channel quads wherever they apply; the channel tile kernel) gives the
    oracle's plane."""
    from paper_2511_02328_gb300.search import Plan
    if kernel in ("pairs", "triples", "quads"):
        monkeypatch.setenv("AFGB_DEDISP_KERNEL", "pairs")
        monkeypatch.setenv("AFGB_PAIR_GROUP", {"pairs": "2", "triples": "3", "quads": "4"}[kernel])
    elif kernel != "auto":
        monkeypatch.setenv("AFGB_DEDISP_KERNEL", kernel)
    nchan, f_lo, f_hi, tsamp, nsamp, dms = shape
    rng = np.random.default_rng(nchan * 7 + nsamp)
    x = rng.integers(0, 256, (nchan, nsamp), dtype=np.uint8)
    D = oracle.delay_table(nchan, f_lo, f_hi, tsamp, dms)
    Y = oracle.dedisperse(x, D)
    p = Plan(nchan, f_lo, f_hi, tsamp, dms)
    plane = p.dedisperse(torch.from_numpy(x).cuda())
    nout = Y.shape[1]
    widths = [w for w in [1, 2, 3, 8, 16] if w <= nout]
    snr, bw = p.boxcar_snr(plane, widths)
    torch.cuda.synchronize()
    assert np.array_equal(plane.cpu().numpy(), Y)
    ref_snr, ref_bw = oracle.boxcar_snr(Y, widths)
    _snr_close(snr.cpu().numpy(), ref_snr)
    p.close()


def test_extreme_values_bit_exact():
    from paper_2511_02328_gb300.search import Plan
    # all-255 input: every plane value is 255*nchan (the int32 range the kernel
    # must hold), and the plane is the oracle's (every path is forced in
    # test_gpu_saturation.py)
    nchan, nsamp = 4096, 4096
    dms = np.arange(0, 16, 1.0)
    p = Plan(nchan, 1000.0, 1500.0, 4.9152e-5, dms)
    x = torch.full((nchan, nsamp), 255, dtype=torch.uint8, device="cuda")
    plane = p.dedisperse(x)
    torch.cuda.synchronize()
    D = oracle.delay_table(nchan, 1000.0, 1500.0, 4.9152e-5, dms)
    Y = oracle.dedisperse(np.full((nchan, nsamp), 255, np.uint8), D)
    assert np.array_equal(plane.cpu().numpy(), Y)
    assert int(Y.min()) == int(Y.max()) == 255 * nchan
    p.close()


def test_boxcar_and_candidates_on_wide_range_planes():
    """Planes whose window deviations |B - q| pass 2^22 in some tiles and not
    in others (the boxcar kernel's two conversion paths), with full-range
    spikes; candidates from a 16-byte aligned and from a misaligned S/N plane."""
    from paper_2511_02328_gb300.search import Plan
    nchan = 4096
    p = Plan(nchan, 1000.0, 1500.0, 4.9152e-5, [0.0, 1.0, 2.0, 3.0, 4.0])
    rng = np.random.default_rng(11)
    ndm, nout = 5, 3 * 4096 + 777
    Y = rng.integers(500_000, 501_000, (ndm, nout)).astype(np.int32)
    Y[1, 5000:5040] = 255 * nchan                      # full-range block: generic path there
    Y[2, 100:103] = 0
    Y[3, ::997] = 255 * nchan                           # isolated spikes in every tile
    Y[4, 9000:9300] += 4_000                            # a broad pulse, fast path
    widths = [1, 2, 4, 8, 16, 32, 64, 128, 256]
    plane = torch.from_numpy(Y).cuda()
    snr, bw = p.boxcar_snr(plane, widths)
    torch.cuda.synchronize()
    ref_snr, ref_bw = oracle.boxcar_snr(Y, widths)
    _snr_close(snr.cpu().numpy(), ref_snr)
    _widths_agree(bw.cpu().numpy(), ref_bw, Y, widths)
    ref, nref = oracle.peaks(ref_snr, ref_bw, widths, 4.0)
    assert nref > 10
    got, n = p.cands_to_numpy(*p.candidates(snr, bw, widths, 4.0))
    _cands_agree(got, ref, ref_snr, 4.0)
    buf = torch.empty(ndm * nout + 1, dtype=torch.float32, device="cuda")
    snr_off = buf[1:].view(ndm, nout)                   # 4-byte offset: scalar loads
    snr_off.copy_(snr)
    assert snr_off.data_ptr() % 16 != 0
    got2, n2 = p.cands_to_numpy(*p.candidates(snr_off, bw, widths, 4.0))
    assert n2 == n and np.array_equal(got2, got)
    p.close()


def test_nout_one_and_width_equal_nout():
    from paper_2511_02328_gb300.search import Plan
    nchan, tsamp = 16, 1e-3
    dms = [0.0, 20.0]
    D = oracle.delay_table(nchan, 1000.0, 1500.0, tsamp, dms)
    nsamp = int(D.max()) + 1
    x = np.random.default_rng(0).integers(0, 256, (nchan, nsamp), dtype=np.uint8)
    p = Plan(nchan, 1000.0, 1500.0, tsamp, dms)
    plane = p.dedisperse(torch.from_numpy(x).cuda())
    snr, bw = p.boxcar_snr(plane, [1])
    torch.cuda.synchronize()
    assert np.array_equal(plane.cpu().numpy(), oracle.dedisperse(x, D))
    assert np.all(snr.cpu().numpy() == 0.0)                 # one sample: sigma = 0
    p.close()


def test_capacity_overflow_reports_total(c1_data):
    x, D, Y, ref_snr, ref_bw = c1_data
    p = _plan(C1)
    from paper_2511_02328_gb300 import _lib
    _lib.af_search_reserve(p.handle, x.shape[1], 2)
    out = np.empty(2, dtype=_lib.CAND_DTYPE)
    cands, n = _lib.af_search(p.handle, x, x.shape[1], C1["widths"], 5.0, 2, out=out)
    ref, nref = oracle.peaks(ref_snr, ref_bw, C1["widths"], 5.0)
    assert nref > 2
    full, nfull = p.search_host(x, C1["widths"], 5.0, cap=1 << 16)
    assert abs(nfull - nref) <= _cands_agree(full, ref, ref_snr, 5.0)
    assert n == nfull and len(cands) == 2
    p.close()


def test_argument_errors():
    from paper_2511_02328_gb300 import _lib
    p = _plan(C1)
    x = torch.zeros((C1["nchan"], 100), dtype=torch.uint8, device="cuda")
    with pytest.raises(_lib.AFError) as e:           # nsamp <= Dmax
        p.dedisperse(x)
    assert e.value.code == _lib.AF_EINVAL
    plane = torch.zeros((p.ndm, 1000), dtype=torch.int32, device="cuda")
    with pytest.raises(_lib.AFError):
        p.boxcar_snr(plane, [4, 2])                   # not ascending
    with pytest.raises(_lib.AFError):
        p.boxcar_snr(plane, [1, 2000])                # wider than nout
    with pytest.raises(_lib.AFError) as e:
        _lib.af_search(p.handle, np.zeros((C1["nchan"], 20000), np.uint8), 20000, [1], 8.0, 16)
    assert e.value.code == _lib.AF_ENOBUFS           # no reservation
    p.close()


@pytest.mark.slow
def test_c2_sampled_rows():
    """Full-size 4096-channel workload in the benchmark's launch
    configuration; plane rows and S/N sampled against the oracle."""
    cfg = C2
    dms = dm_list(cfg)
    rng = np.random.default_rng(2)
    pulses = []
    D = oracle.delay_table(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms)
    for k in range(5):
        dm0 = float(rng.uniform(50, 1000))
        t0 = int(rng.integers(1000, 200000))
        offs = oracle.injection_offsets(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dm0, t0)
        pulses.append(synth.Pulse(offs, 20, synth.pulse_amplitude(20.0, cfg["nchan"], 20)))
    x = synth.filterbank(cfg["nchan"], cfg["nsamp"], seed=2, pulses=pulses)
    p = _plan(cfg)
    p.reserve(cfg["nsamp"])
    assert p.kernel()["path"] == "pairs"        # the benchmark's path on this workload
    stats = torch.empty((p.ndm, 2), dtype=torch.int64, device="cuda")
    plane = p.dedisperse(torch.from_numpy(x).cuda(), stats=stats)
    snr, bw = p.boxcar_snr(plane, cfg["widths"], stats=stats)
    torch.cuda.synchronize()
    rows = sorted(set([0, 1, 499, 500, len(dms) - 1] + rng.integers(0, len(dms), 6).tolist()))
    Yr = oracle.dedisperse(x, D[rows], nout=plane.shape[1])
    got = plane[rows].cpu().numpy()
    assert np.array_equal(got, Yr)
    ref_snr, ref_bw = oracle.boxcar_snr(Yr, cfg["widths"])
    _snr_close(snr[rows].cpu().numpy(), ref_snr)
    p.close()


def test_fallback_kernel_for_wide_delay_spread():
    """A DM grid so coarse that a block's delay spread does not fit the
    shared-memory window runs on the fallback kernel; still bit-exact."""
    from paper_2511_02328_gb300.search import Plan
    nchan, tsamp = 64, 1e-4
    dms = [0.0, 3000.0, 6000.0]
    D = oracle.delay_table(nchan, 1000.0, 1500.0, tsamp, dms)
    nsamp = int(D.max()) + 3000
    x = np.random.default_rng(4).integers(0, 256, (nchan, nsamp), dtype=np.uint8)
    p = Plan(nchan, 1000.0, 1500.0, tsamp, dms)
    assert p.kernel()["path"] == "simple"
    plane = p.dedisperse(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(plane.cpu().numpy(), oracle.dedisperse(x, D))
    p.close()


def _expected_ring(spread, nw=11, m=8):
    """Deepest ring (4, 3, 2) whose shared memory fits the device's opt-in
    limit: ring x (32 channel windows of rw bytes + the offset tables + 2 barriers)."""
    optin = getattr(torch.cuda.get_device_properties(0), "shared_memory_per_block_optin", 232448)
    rw = (15 + spread + 128 * m + 15) & ~15
    for ns in (4, 3, 2):
        if ns * 32 * rw + ns * nw * 48 * 4 + 16 * ns <= optin:
            return ns
    return 0


@pytest.mark.parametrize("step,ring", [(1.0, 4), (4.0, 3), (5.0, 3), (6.0, 2), (10.0, 2), (12.0, 0)])
def test_coarse_dm_grids_shallower_ring(step, ring, monkeypatch):
    """Coarse DM grids widen each channel's window; the tile kernel then runs
    with a 3- or 2-deep ring before the fallback kernel takes over.  Every
    depth gives the oracle's plane and row sums bit-exact (256 channels,
    1000-1500 MHz, 98.304 us, 61 DMs of the given step, a ragged last tile)."""
    from paper_2511_02328_gb300.search import Plan
    monkeypatch.setenv("AFGB_DEDISP_KERNEL", "tile")
    nchan, tsamp = 256, 98.304e-6
    dms = np.arange(0.0, 1.0 + 60 * step, step)
    D = oracle.delay_table(nchan, 1000.0, 1500.0, tsamp, dms)
    nsamp = int(D.max()) + 3 * 8192 + 77
    x = np.random.default_rng(int(step * 10)).integers(0, 256, (nchan, nsamp), dtype=np.uint8)
    p = Plan(nchan, 1000.0, 1500.0, tsamp, dms)
    k = p.kernel()
    assert k["ring"] == _expected_ring(k["spread"]) == ring
    assert k["path"] == ("tile" if ring else "simple")
    stats = torch.empty((p.ndm, 2), dtype=torch.int64, device="cuda")
    plane = p.dedisperse(torch.from_numpy(x).cuda(), stats=stats)
    torch.cuda.synchronize()
    Y = oracle.dedisperse(x, D)
    assert np.array_equal(plane.cpu().numpy(), Y)
    S, Q = oracle.rowstats(Y)
    st = stats.cpu().numpy()
    assert np.array_equal(st[:, 0], S) and np.array_equal(st[:, 1], Q)
    p.close()


def _pair_rows_bytes(D, L, G=2):
    """Bytes of the group-row buffer for time blocks of L outputs: per group
    q (channels Gq .. Gq+G-1) one row per distinct tuple of delays relative
    to channel Gq (0 for a missing channel), each of r16(L + 2 span + 32)
    uint16 samples, span = the largest D[.][Gq] of the DMs with that tuple
    minus their smallest rounded down to 16."""
    ndm, nchan = D.shape
    total = 0
    for q in range((nchan + G - 1) // G):
        c0 = G * q
        rel = np.stack([D[:, c0 + i] - D[:, c0] if c0 + i < nchan else np.zeros(ndm, dtype=D.dtype)
                        for i in range(1, G)], axis=1)
        for v in np.unique(rel, axis=0):
            d0 = D[np.all(rel == v, axis=1), c0]
            span = int(d0.max()) - (int(d0.min()) & ~15)
            total += (L + 2 * span + 32 + 15) & ~15
    return 2 * total


@pytest.mark.parametrize("G", [2, 3, 4])
@pytest.mark.parametrize("nchan,f_lo,f_hi", [(256, 1000.0, 1500.0), (255, 1500.0, 1000.0)])
def test_pair_rows_several_time_blocks(nchan, f_lo, f_hi, G, monkeypatch):
    """The group-row path (2, 3, 4 channels) with a row budget that holds 9 tiles
    of outputs: the plane (several time blocks, a ragged last one) and its row
    sums are the oracle's; 255 channels end with a short group."""
    from paper_2511_02328_gb300.search import Plan
    tsamp, dms = 98.304e-6, np.arange(0.0, 301.0, 1.0)
    D = oracle.delay_table(nchan, f_lo, f_hi, tsamp, dms)
    nsamp = int(D.max()) + 30 * 1016 + 311
    budget = _pair_rows_bytes(D, 9 * 1016, G)
    assert budget < _pair_rows_bytes(D, 31 * 1016, G)
    monkeypatch.setenv("AFGB_PAIR_BUDGET_MB", str(-(-budget // (1 << 20))))
    monkeypatch.setenv("AFGB_DEDISP_KERNEL", "pairs")
    monkeypatch.setenv("AFGB_PAIR_GROUP", str(G))
    x = np.random.default_rng(nchan).integers(0, 256, (nchan, nsamp), dtype=np.uint8)
    p = Plan(nchan, f_lo, f_hi, tsamp, dms)
    assert p.kernel()["path"] == "tile"                 # nothing reserved yet
    p.reserve(nsamp)
    assert (p.kernel()["path"], p.kernel()["group"]) == ("pairs", G)
    stats = torch.empty((p.ndm, 2), dtype=torch.int64, device="cuda")
    plane = p.dedisperse(torch.from_numpy(x).cuda(), stats=stats)
    torch.cuda.synchronize()
    Y = oracle.dedisperse(x, D)
    assert np.array_equal(plane.cpu().numpy(), Y)
    S, Q = oracle.rowstats(Y)
    st = stats.cpu().numpy()
    assert np.array_equal(st[:, 0], S) and np.array_equal(st[:, 1], Q)
    p.close()


def test_pair_rows_forced_and_default_choice(c1_data, monkeypatch):
    """AFGB_DEDISP_KERNEL=pairs puts the 256-channel workload on group rows;
    without it the reservation keeps whichever path its cost model prefers,
    and both give the oracle's plane."""
    x, D, Y, _, _ = c1_data
    for k in ("pairs", None):
        if k:
            monkeypatch.setenv("AFGB_DEDISP_KERNEL", k)
        else:
            monkeypatch.delenv("AFGB_DEDISP_KERNEL", raising=False)
        p = _plan(C1)
        p.reserve(x.shape[1])
        path = p.kernel()["path"]
        assert path == "pairs" if k else path in ("pairs", "tile")
        plane = p.dedisperse(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(plane.cpu().numpy(), Y)
        p.close()


def test_simple_kernel_forced_matches(c1_data, monkeypatch):
    """The fallback kernel selected explicitly gives the same plane."""
    from paper_2511_02328_gb300.search import Plan
    x, D, Y, _, _ = c1_data
    monkeypatch.setenv("AFGB_DEDISP_KERNEL", "simple")
    p = _plan(C1)
    k = p.kernel()
    assert (k["path"], k["ring"], k["group"]) == ("simple", 0, 1)
    stats = torch.empty((p.ndm, 2), dtype=torch.int64, device="cuda")
    plane = p.dedisperse(torch.from_numpy(x).cuda(), stats=stats)
    torch.cuda.synchronize()
    assert np.array_equal(plane.cpu().numpy(), Y)
    S, Q = oracle.rowstats(Y)
    assert np.array_equal(stats.cpu().numpy()[:, 0], S)
    p.close()


def test_repeated_calls_and_streams(c1_data):
    """Same plan, two streams used one after the other, repeated calls: identical planes."""
    x, D, Y, _, _ = c1_data
    p = _plan(C1)
    xd = torch.from_numpy(x).cuda()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a = p.dedisperse(xd, stream=s1)
    s1.synchronize()
    b = p.dedisperse(xd, stream=s2)
    s2.synchronize()
    assert np.array_equal(a.cpu().numpy(), Y) and np.array_equal(b.cpu().numpy(), Y)
    p.close()


def test_plans_with_different_windows_coexist(c1_data):
    """A plan created later with a smaller shared-memory window must not break
    an earlier plan that needs a larger one (the limit belongs to the kernel)."""
    from paper_2511_02328_gb300.search import Plan
    x, D, Y, _, _ = c1_data
    big = _plan(C1)                                           # 501 DMs, wide window
    small = Plan(C1["nchan"], C1["f_lo"], C1["f_hi"], C1["tsamp"], [0.0, 0.5])
    plane = big.dedisperse(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(plane.cpu().numpy(), Y)
    small.close()
    big.close()


def test_diag_int_rates_plausible():
    # the measured integer rates that the bench's roofline reports: positive,
    # below the nominal 128 lanes x 2.07 GHz per SM, and the dedispersion step
    # no faster than plain additions
    from paper_2511_02328_gb300 import _lib
    add, pattern = _lib.af_diag_int_rates()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = nsm * 128 * 2.07e9
    assert 0.1 * nominal < add <= 1.05 * nominal
    assert 0.05 * nominal < pattern <= 1.05 * add


def test_diag_smem_rate_plausible():
    # the measured shared-memory load bandwidth (the group-row tile kernel's
    # roofline denominator): positive and at most 128 B per SM per clock at
    # the 2.07 GHz maximum clock
    from paper_2511_02328_gb300 import _lib
    bw = _lib.af_diag_smem_rate()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = nsm * 128 * 2.07e9
    assert 0.2 * nominal < bw <= 1.05 * nominal


def test_workspace_sizes_match_reservations(c1_data):
    """af_dedisperse_workspace_size / af_search_workspace_size report what the
    reservations then take from the device (allocation granularity aside),
    without allocating themselves."""
    from paper_2511_02328_gb300 import _lib
    x, D, Y, _, _ = c1_data
    nsamp = x.shape[1]
    p = _plan(C1)
    torch.cuda.synchronize()
    f0 = torch.cuda.mem_get_info()[0]
    want = _lib.af_dedisperse_workspace_size(p.handle, nsamp)
    assert torch.cuda.mem_get_info()[0] == f0
    _lib.af_dedisperse_reserve(p.handle, nsamp)
    used = f0 - torch.cuda.mem_get_info()[0]
    assert want <= used <= want + (64 << 20)
    assert (want > 0) == (p.kernel()["path"] == "pairs")
    q = _plan(C1)
    s_want = _lib.af_search_workspace_size(q.handle, nsamp, 1024)
    f1 = torch.cuda.mem_get_info()[0]
    _lib.af_search_reserve(q.handle, nsamp, 1024)
    s_used = f1 - torch.cuda.mem_get_info()[0]
    assert s_want <= s_used <= s_want + (128 << 20)
    with pytest.raises(_lib.AFError):
        _lib.af_dedisperse_workspace_size(p.handle, int(D.max()))     # nsamp <= Dmax
    p.close()
    q.close()


def test_cluster_equals_the_oracle_rule():
    """af_cluster against the oracle's greedy rule (Sec. 4.2 tolerances: |dDM| < 20,
    |dTOA| < 0.2 s) on random candidate lists with many equal S/N values: the same
    clusters are kept, in the same order."""
    from oracle import nms
    from paper_2511_02328_gb300 import _lib
    dms = dm_list(C1)
    p = _plan(C1)
    rng = np.random.default_rng(11)
    span = 30000
    for n in (0, 1, 2, 50, 400, 2000):
        key = rng.choice(len(dms) * span, size=n, replace=False)   # distinct (dm_idx, t)
        a = np.zeros(n, dtype=_lib.CAND_DTYPE)
        a["dm_idx"] = key // span
        a["t"] = key % span
        a["abs_sample"] = a["t"]
        a["width"] = 1 << rng.integers(0, 6, n)
        a["snr"] = rng.choice(np.arange(6.0, 30.0, 0.5), n)
        kept = p.cluster(a.copy())
        ref = nms.cluster([(int(c["dm_idx"]), int(c["t"]), int(c["width"]), float(c["snr"])) for c in a],
                          dms, C1["tsamp"])
        assert [(int(c["dm_idx"]), int(c["t"])) for c in kept] == [(c[0], c[1]) for c in ref], n
    p.close()
