"""Saturating and adversarial 8-bit inputs on every dedispersion path that
keeps partial sums in 16-bit lanes, compared element by element with the
oracle's brute-force plane (Sec. 2.3: Y[d][t] = sum_c X[c][t + D[d][c]]).

The lanes are exact only because each kernel folds them into 32-bit sums
before they can reach 2^16:
  - group rows of G channels (2, 3, 4): at most 65535 / (255 G) rows between
    folds, i.e. 128, 85 and 64 rows;
  - the channel tile kernel (single plans, the persistent batch kernel, the
    streaming engine's tile path): 256 channels between folds;
  - subband stage 1: uint16 partial sums for subbands of up to 257 channels
    (257 * 255 = 65535).
All-255 input drives every lane to its largest value right before each fold
(one row or channel too many would wrap), and the mixed patterns (255/0 by
channel, by sample parity, in channel blocks of a fold's length, near-255
noise) make the lanes of one word differ, so that a lane carry, a wrong
bucket or a misaligned offset shows.  Shapes span several folds (>= 256
channels), several DM blocks and several time tiles with a ragged tail."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def pattern(kind, nchan, nsamp, seed=0):
    """uint8 [nchan][nsamp] test inputs (no search arithmetic)."""
    rng = np.random.default_rng(seed)
    c = np.arange(nchan)[:, None]
    t = np.arange(nsamp)[None, :]
    if kind == "full":
        return np.full((nchan, nsamp), 255, np.uint8)
    if kind == "alt_chan":               # 255 / 0 per channel
        return np.broadcast_to(np.where(c % 2 == 0, 255, 0), (nchan, nsamp)).astype(np.uint8)
    if kind == "alt_time":               # 255 / 0 by the parity of c + t: the two lanes of a word differ
        return np.where((c + t) % 2 == 0, 255, 0).astype(np.uint8)
    if kind == "fold_blocks":            # fold-length blocks of saturated channels between random ones
        x = rng.integers(0, 256, (nchan, nsamp), dtype=np.uint8)
        x[(np.arange(nchan) // 256) % 2 == 0] = 255
        return x
    if kind == "near_full":              # 255 except sparse 0..3 dips: saturated but not uniform
        x = np.full((nchan, nsamp), 255, np.uint8)
        m = rng.random((nchan, nsamp)) < 0.05
        x[m] = rng.integers(0, 4, int(m.sum()), dtype=np.uint8)
        return x
    if kind == "binary":                 # 255 with p = 0.9, else 0
        return np.where(rng.random((nchan, nsamp)) < 0.9, 255, 0).astype(np.uint8)
    raise ValueError(kind)


KINDS = ["full", "alt_chan", "alt_time", "fold_blocks", "near_full", "binary"]

# 1024 channels (4-12 folds of every lane kind), DMs 0..60 (5 blocks of 15,
# 6 of 11), 1000-1500 MHz at 98.304 us: Dmax = 1406, nout = 5011 (4 tiles + a
# ragged tail)
NCHAN, F_LO, F_HI, TSAMP = 1024, 1000.0, 1500.0, 98.304e-6
DMS = np.arange(0.0, 61.0, 1.0)


def _env(monkeypatch, kernel=None, group=None):
    for k in ("AFGB_DEDISP_KERNEL", "AFGB_PAIR_GROUP"):
        monkeypatch.delenv(k, raising=False)
    if kernel:
        monkeypatch.setenv("AFGB_DEDISP_KERNEL", kernel)
    if group:
        monkeypatch.setenv("AFGB_PAIR_GROUP", str(group))


@pytest.fixture(scope="module")
def delays():
    return oracle.delay_table(NCHAN, F_LO, F_HI, TSAMP, DMS)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("path", ["pairs2", "pairs3", "pairs4", "tile", "simple"])
def test_single_plan_paths(path, kind, delays, monkeypatch):
    """Group rows of 2, 3 and 4 channels (forced, reserved), the channel tile
    kernel and the fallback kernel: plane and row sums equal the oracle's."""
    from paper_2511_02328_gb300.search import Plan
    D = delays
    nsamp = int(D.max()) + 5011
    if path.startswith("pairs"):
        _env(monkeypatch, "pairs", int(path[-1]))
    else:
        _env(monkeypatch, path)
    x = pattern(kind, NCHAN, nsamp, seed=len(kind))
    p = Plan(NCHAN, F_LO, F_HI, TSAMP, DMS)
    if path.startswith("pairs"):
        p.reserve(nsamp)
        assert (p.kernel()["path"], p.kernel()["group"]) == ("pairs", int(path[-1]))
    else:
        assert p.kernel()["path"] == path
    stats = torch.empty((p.ndm, 2), dtype=torch.int64, device="cuda")
    plane = p.dedisperse(torch.from_numpy(x).cuda(), stats=stats)
    torch.cuda.synchronize()
    Y = oracle.dedisperse(x, D)
    got = plane.cpu().numpy()
    assert got.shape == Y.shape
    bad = np.argwhere(got != Y)
    assert bad.size == 0, (path, kind, bad[:5].tolist(), got[tuple(bad[0])], Y[tuple(bad[0])])
    S, Q = oracle.rowstats(Y)
    st = stats.cpu().numpy()
    assert np.array_equal(st[:, 0], S) and np.array_equal(st[:, 1], Q)
    p.close()


@pytest.mark.parametrize("G", [2, 3, 4])
def test_group_rows_several_time_blocks_saturated(G, delays, monkeypatch):
    """Group rows in several time blocks (a row budget of about 9 of the 26
    output tiles) on all-255, near-255 and parity-alternating input: the fold
    counts hold in every block."""
    from paper_2511_02328_gb300.search import Plan
    from paper_2511_02328_gb300 import _lib
    D = delays
    nsamp = int(D.max()) + 25 * 1016 + 333
    _env(monkeypatch, "pairs", G)
    p0 = Plan(NCHAN, F_LO, F_HI, TSAMP, DMS)
    nine = _lib.af_dedisperse_workspace_size(p0.handle, int(D.max()) + 9 * 1016)   # rows of 9 tiles
    assert 0 < nine < _lib.af_dedisperse_workspace_size(p0.handle, int(D.max()) + 12 * 1016)
    p0.close()
    monkeypatch.setenv("AFGB_PAIR_BUDGET_MB", str(-(-nine // (1 << 20))))
    for kind in ("full", "near_full", "alt_time"):
        x = pattern(kind, NCHAN, nsamp, seed=G)
        p = Plan(NCHAN, F_LO, F_HI, TSAMP, DMS)
        p.reserve(nsamp)
        assert (p.kernel()["path"], p.kernel()["group"]) == ("pairs", G)
        plane = p.dedisperse(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(plane.cpu().numpy(), oracle.dedisperse(x, D)), kind
        p.close()


def test_all_255_at_4096_channels_every_path(monkeypatch):
    """The benchmark's channel count (4096, 16 folds of the tile kernel's
    lanes, 48-64 of the group rows'): all-255 input on every path gives
    the oracle's plane (255 * 4096 everywhere), not just a constant one."""
    from paper_2511_02328_gb300.search import Plan
    nchan, tsamp = 4096, 49.152e-6
    dms = np.arange(0.0, 31.0, 1.0)
    D = oracle.delay_table(nchan, F_LO, F_HI, tsamp, dms)
    nsamp = int(D.max()) + 3 * 1016 + 5
    for kind in ("full", "near_full"):
        x = pattern(kind, nchan, nsamp, seed=7)
        Y = oracle.dedisperse(x, D)
        if kind == "full":
            assert int(Y.min()) == int(Y.max()) == 255 * nchan
        xd = torch.from_numpy(x).cuda()
        for path in ("pairs2", "pairs3", "pairs4", "tile", "simple"):
            if path.startswith("pairs"):
                _env(monkeypatch, "pairs", int(path[-1]))
            else:
                _env(monkeypatch, path)
            p = Plan(nchan, F_LO, F_HI, tsamp, dms)
            if path.startswith("pairs"):
                p.reserve(nsamp)
                assert p.kernel()["path"] == "pairs"
            plane = p.dedisperse(xd)
            torch.cuda.synchronize()
            assert np.array_equal(plane.cpu().numpy(), Y), (kind, path)
            p.close()


@pytest.mark.parametrize("kind", ["full", "alt_time", "near_full", "fold_blocks"])
@pytest.mark.parametrize("nchan,nsub", [(514, 2), (1028, 4), (768, 3)])
def test_subband_stage1_uint16_at_its_limit(nchan, nsub, kind):
    """Subbands of 257 channels (uint16 partial sums reach exactly 65535 on
    all-255 input) and of 256: the two-stage plane equals the oracle's
    subband definition (Sec. 2.3, Eqs. stage1, residual, stage2)."""
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import Plan
    dms = np.arange(0.0, 97.0, 1.0)
    n0 = 8
    tab = oracle.subband_tables(nchan, F_LO, F_HI, TSAMP, dms, n0, nsub, oracle.FS_INVSQ)
    sizes = np.diff(tab["first"])
    assert sizes.max() == (257 if nchan % 257 == 0 else 256)
    nsamp = int(oracle.subband_effective_delays(tab).max()) + 4 * 1020 + 77
    x = pattern(kind, nchan, nsamp, seed=nchan)
    Yref = oracle.subband_dedisperse(x, tab)
    p = Plan(nchan, F_LO, F_HI, TSAMP, dms, subband=dict(n0=n0, nsub=nsub, fs_mode=_lib.AF_FS_INVSQ))
    stats = torch.empty((p.ndm, 2), dtype=torch.int64, device="cuda")
    plane = p.dedisperse(torch.from_numpy(x).cuda(), stats=stats)
    torch.cuda.synchronize()
    _lib.af_plan_check(p.handle)
    assert np.array_equal(plane.cpu().numpy(), Yref)
    S, Q = oracle.rowstats(Yref)
    st = stats.cpu().numpy()
    assert np.array_equal(st[:, 0], S) and np.array_equal(st[:, 1], Q)
    p.close()


BATCH_BEAMS = [
    # nchan, f_lo, f_hi, tsamp, nsamp, dms, widths, thresh, kind
    (1024, 1000.0, 1500.0, 98.304e-6, 6500, np.arange(0.0, 61.0, 1.0), [1, 4], 6.0, "full"),
    (512, 1500.0, 1000.0, 98.304e-6, 6000, np.arange(0.0, 50.0, 0.5), [1, 2], 6.0, "alt_time"),
    (771, 1000.0, 1500.0, 98.304e-6, 7000, np.arange(0.0, 40.0, 1.0), [1, 8], 6.0, "near_full"),
    (256, 1000.0, 1500.0, 98.304e-6, 9000, np.arange(0.0, 120.0, 2.0), [2, 4], 6.0, "binary"),
]


@pytest.mark.parametrize("strategy", ["tile", "pairs", "persistent"])
def test_batch_strategies_saturated(strategy, monkeypatch):
    """The batch's persistent channel-tile kernel, its beam-after-beam group
    rows and its persistent group rows on saturated and mixed beams: every
    beam's plane is the oracle's."""
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import device_view
    _env(monkeypatch, "pairs" if strategy != "tile" else None)
    monkeypatch.setenv("AFGB_BATCH_STRATEGY", strategy)
    xs = [pattern(b[8], b[0], b[4], seed=i) for i, b in enumerate(BATCH_BEAMS)]
    xs_dev = [torch.from_numpy(x).cuda() for x in xs]
    descs = [dict(nchan=b[0], f_lo=b[1], f_hi=b[2], tsamp=b[3], dm_list=b[5], d_in=xd.data_ptr(), nsamp=b[4],
                  widths=b[6], thresh=b[7], cap=1 << 12) for b, xd in zip(BATCH_BEAMS, xs_dev)]
    batch = _lib.af_batch_build(descs, 0)
    _lib.af_batch_run(batch, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for i, (b, x) in enumerate(zip(BATCH_BEAMS, xs)):
        pl, sn, bw, nout = _lib.af_batch_buffers(batch, i)
        plane = device_view(pl, (len(b[5]), nout), torch.int32).cpu().numpy()
        D = oracle.delay_table(b[0], b[1], b[2], b[3], b[5])
        assert np.array_equal(plane, oracle.dedisperse(x, D)), (strategy, i)
    _lib.af_batch_destroy(batch)


@pytest.mark.parametrize("kernel", ["pairs", "tile"])
def test_stream_windows_saturated(kernel, monkeypatch):
    """The streaming engine on saturated and mixed chunks (group rows forced,
    the persistent channel-tile kernel forced): concatenated window planes
    equal the oracle's plane of the whole stream."""
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import device_view
    _env(monkeypatch, kernel)
    nchan, dms, window, nwin = 512, np.arange(0.0, 46.0, 1.0), 4096, 4
    D = oracle.delay_table(nchan, F_LO, F_HI, TSAMP, dms)
    hop = window - int(D.max())
    total = window + (nwin - 1) * hop
    x = pattern("near_full", nchan, total, seed=5)
    x[:, window:window + hop] = pattern("alt_time", nchan, hop)
    x[:, window + hop:window + 2 * hop] = 255
    s = _lib.af_stream_open(1, nchan, F_LO, F_HI, TSAMP, dms, window, [1, 2, 4], 6.0, 1 << 12)
    planes = []
    for k in range(nwin):
        chunk = x[:, :window] if k == 0 else x[:, window + (k - 1) * hop: window + k * hop]
        _lib.af_stream_push(s, 0, chunk, k)
        r = _lib.af_stream_poll(s, 60000)
        assert r is not None and r["seq"] == k
        pl, sn, nout = _lib.af_stream_result_plane(s, r["slot"])
        planes.append(device_view(pl, (len(dms), nout), torch.int32).cpu().numpy())
        _lib.af_stream_release(s, r["slot"])
    _lib.af_stream_close(s)
    assert np.array_equal(np.concatenate(planes, axis=1), oracle.dedisperse(x, D))
