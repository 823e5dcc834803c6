"""Streaming engine: windows overlapping by Dmax tile the stream exactly
(concatenated planes equal the one-shot plane, bit-exact); each beam's result
is the same alone and in a mix of concurrently processed beams; slots are
admitted by the HBM budget; host-injected faults (dropped, repeated or
mis-sized chunks, a beam that stops) are rejected without disturbing other
beams; a snapshot restored into a fresh engine continues exactly; p50/p99
latency is reported."""
import numpy as np
import pytest

import oracle
from paper_2511_02328_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NCHAN, F_LO, F_HI, TSAMP = 64, 1000.0, 1500.0, 5e-4
DMS = np.arange(0.0, 41.0, 1.0)
WINDOW = 4096
WIDTHS = [1, 2, 4, 8]
THRESH = 6.0
NWIN = 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _dmax():
    return int(oracle.delay_table(NCHAN, F_LO, F_HI, TSAMP, DMS).max())


def _stream_data(seed):
    dmax = _dmax()
    hop = WINDOW - dmax
    total = WINDOW + (NWIN - 1) * hop
    pulses = []
    rng = np.random.default_rng(seed)
    for k in range(NWIN):
        t0 = k * hop + int(rng.integers(100, hop - 100))
        offs = oracle.injection_offsets(NCHAN, F_LO, F_HI, TSAMP, float(rng.integers(5, 35)), t0)
        pulses.append(synth.Pulse(offs, 2, synth.pulse_amplitude(20.0, NCHAN, 2)))
    return synth.filterbank(NCHAN, total, seed=seed, pulses=pulses), hop


def _chunk(x, k, hop):
    # column slices of the stream: passed to the engine with their row pitch
    if k == 0:
        return x[:, :WINDOW]
    return x[:, WINDOW + (k - 1) * hop: WINDOW + k * hop]


def _open(nbeams, **kw):
    from paper_2511_02328_gb300 import _lib
    return _lib.af_stream_open(nbeams, NCHAN, F_LO, F_HI, TSAMP, DMS, WINDOW, WIDTHS, THRESH, 1 << 12, **kw)


def _drain(s, n, keep_planes=False):
    """Poll n results; returns {(beam, seq): (result, plane or None)}."""
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import device_view
    out = {}
    for _ in range(n):
        r = _lib.af_stream_poll(s, 60000)
        assert r is not None, "no result"
        plane = None
        if keep_planes:
            pl, sn, nout = _lib.af_stream_result_plane(s, r["slot"])
            plane = device_view(pl, (len(DMS), nout), torch.int32).cpu().numpy()
        _lib.af_stream_release(s, r["slot"])
        out[(r["beam"], r["seq"])] = (r, plane)
    return out


@pytest.mark.parametrize("kernel", ["auto", "pairs", "tile"])
def test_concatenated_windows_equal_one_shot(kernel, monkeypatch):
    """On every dedispersion path of the engine (its default choice, group rows
    forced, the persistent channel-tile kernel forced)."""
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import Plan
    if kernel != "auto":
        monkeypatch.setenv("AFGB_DEDISP_KERNEL", kernel)
    x, hop = _stream_data(1)
    s = _open(1)
    h, dmax, nslots = _lib.af_stream_info(s)
    assert h == hop and dmax == _dmax()
    res = {}
    for k in range(NWIN):
        _lib.af_stream_push(s, 0, _chunk(x, k, hop), k)
        res.update(_drain(s, 1, keep_planes=True))
    _lib.af_stream_close(s)
    planes = np.concatenate([res[(0, k)][1] for k in range(NWIN)], axis=1)
    D = oracle.delay_table(NCHAN, F_LO, F_HI, TSAMP, DMS)
    assert np.array_equal(planes, oracle.dedisperse(x, D))
    # each window's candidates are those of the same window searched alone
    p = Plan(NCHAN, F_LO, F_HI, TSAMP, DMS)
    found = 0
    for k in range(NWIN):
        r = res[(0, k)][0]
        assert r["sample0"] == k * hop
        win = np.ascontiguousarray(x[:, k * hop: k * hop + WINDOW])
        ref, n = p.search_host(win, WIDTHS, THRESH, cap=1 << 12)
        assert r["total"] == n
        assert np.array_equal(r["cands"]["t"], ref["t"]) and np.array_equal(r["cands"]["dm_idx"], ref["dm_idx"])
        assert np.array_equal(r["cands"]["abs_sample"], ref["t"].astype(np.int64) + k * hop)
        found += n
    assert found >= NWIN   # every window holds an injected pulse
    p.close()


def test_alone_equals_in_the_mix():
    from paper_2511_02328_gb300 import _lib
    data = [_stream_data(10 + b) for b in range(3)]
    hop = data[0][1]
    # beam 0 alone
    s = _open(1)
    alone = {}
    for k in range(NWIN):
        _lib.af_stream_push(s, 0, _chunk(data[0][0], k, hop), k)
        alone.update(_drain(s, 1, keep_planes=True))
    _lib.af_stream_close(s)
    # three beams interleaved, several windows in flight at once
    s = _open(3, max_slots=6)
    mix = {}
    for k in range(NWIN):
        for b in range(3):
            _lib.af_stream_push(s, b, _chunk(data[b][0], k, hop), k)
        mix.update(_drain(s, 3, keep_planes=True))
    st = _lib.af_stream_stats(s)
    _lib.af_stream_close(s)
    for k in range(NWIN):
        a, pa = alone[(0, k)]
        m, pm = mix[(0, k)]
        assert np.array_equal(pa, pm)
        assert np.array_equal(a["cands"], m["cands"]) and a["total"] == m["total"]
    assert st["windows"] == 3 * NWIN
    assert st["max_inflight"] >= 2
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert st["rate"] > 0


def test_admission_by_budget():
    from paper_2511_02328_gb300 import _lib
    x, hop = _stream_data(3)
    dmax = _dmax()
    slot_bytes = NCHAN * WINDOW + len(DMS) * hop * 9 + len(DMS) * 16 + (1 << 12) * 24 + 64
    budget = 2 * NCHAN * dmax + slot_bytes + slot_bytes // 2       # room for one slot only
    s = _open(2, hbm_budget=budget, max_slots=8, timeout_ms=0)
    assert _lib.af_stream_info(s)[2] == 1
    _lib.af_stream_push(s, 0, _chunk(x, 0, hop), 0)
    with pytest.raises(_lib.AFError) as e:
        _lib.af_stream_push(s, 1, _chunk(x, 0, hop), 0)       # the only slot is busy
    assert e.value.code == _lib.AF_EAGAIN
    r = _lib.af_stream_poll(s, 60000)
    _lib.af_stream_release(s, r["slot"])
    _lib.af_stream_push(s, 1, _chunk(x, 0, hop), 0)             # admitted once the slot is free
    r = _lib.af_stream_poll(s, 60000)
    assert r["beam"] == 1
    _lib.af_stream_release(s, r["slot"])
    _lib.af_stream_close(s)
    with pytest.raises(_lib.AFError) as e:
        _open(2, hbm_budget=1000)
    assert e.value.code == _lib.AF_ENOBUFS


def test_faults_are_rejected_and_isolated():
    from paper_2511_02328_gb300 import _lib
    x, hop = _stream_data(4)
    s = _open(2)
    _lib.af_stream_push(s, 0, _chunk(x, 0, hop), 0)
    _lib.af_stream_push(s, 1, _chunk(x, 0, hop), 0)
    _drain(s, 2)
    for bad in [(_chunk(x, 2, hop), 2), (_chunk(x, 0, hop), 0), (_chunk(x, 1, hop)[:, :-5], 1)]:
        with pytest.raises(_lib.AFError) as e:      # dropped, repeated, short
            _lib.af_stream_push(s, 0, bad[0], bad[1])
        assert e.value.code == _lib.AF_EINVAL
    with pytest.raises(_lib.AFError):
        _lib.af_stream_push(s, 5, _chunk(x, 1, hop), 1)  # no such beam
    # beam 1 stops sending; beam 0 continues normally
    for k in range(1, NWIN):
        _lib.af_stream_push(s, 0, _chunk(x, k, hop), k)
    res = _drain(s, NWIN - 1)
    assert sorted(res) == [(0, k) for k in range(1, NWIN)]
    _lib.af_stream_close(s)


def test_snapshot_restore_continues_exactly():
    from paper_2511_02328_gb300 import _lib
    x, hop = _stream_data(5)
    dmax = _dmax()
    full = _open(1)
    ref = {}
    for k in range(NWIN):
        _lib.af_stream_push(full, 0, _chunk(x, k, hop), k)
        ref.update(_drain(full, 1, keep_planes=True))
    _lib.af_stream_close(full)
    a = _open(1)
    for k in range(3):
        _lib.af_stream_push(a, 0, _chunk(x, k, hop), k)
        _drain(a, 1)
    ov, nseq, nsample = _lib.af_stream_snapshot(a, 0, NCHAN, dmax)
    _lib.af_stream_close(a)
    assert nseq == 3 and nsample == 3 * hop
    b = _open(1)
    _lib.af_stream_restore(b, 0, ov, nseq, nsample)
    got = {}
    for k in range(3, NWIN):
        _lib.af_stream_push(b, 0, _chunk(x, k, hop), k)
        got.update(_drain(b, 1, keep_planes=True))
    _lib.af_stream_close(b)
    for k in range(3, NWIN):
        assert np.array_equal(got[(0, k)][1], ref[(0, k)][1])
        assert np.array_equal(got[(0, k)][0]["cands"], ref[(0, k)][0]["cands"])


def test_inline_classification_matches_classify():
    """af_stream_classify on a held window equals af_classify on the same window
    searched alone (same cut-outs, same network)."""
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import Plan
    x, hop = _stream_data(6)
    s = _open(1)
    m = _lib.af_model_create(8, 2)
    _lib.af_stream_push(s, 0, _chunk(x, 0, hop), 0)
    r = _lib.af_stream_poll(s, 60000)
    reps = _lib.af_stream_cluster(s, r["cands"])
    assert len(reps) >= 1
    prob = _lib.af_stream_classify(s, r["slot"], m, reps)
    _lib.af_stream_release(s, r["slot"])
    _lib.af_stream_close(s)
    p = Plan(NCHAN, F_LO, F_HI, TSAMP, DMS)
    win = torch.from_numpy(np.ascontiguousarray(x[:, :WINDOW])).cuda()
    plane = p.dedisperse(win)
    cd = torch.from_numpy(np.ascontiguousarray(reps).view(np.uint8).reshape(len(reps), 24)).cuda()
    ref = torch.empty(len(reps), dtype=torch.float32, device="cuda")
    _lib.af_classify(m, p.handle, win.data_ptr(), WINDOW, plane.data_ptr(), plane.shape[1], cd.data_ptr(),
                     len(reps), ref.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(prob, ref.cpu().numpy())
    _lib.af_model_destroy(m)
    p.close()
