"""Many uneven beams in one persistent launch, replayed as a CUDA graph:
every beam's plane is bit-exact with the oracle and with the single-beam
path, its S/N within tolerance, its candidates identical to the single-beam
path; graph replays see new input data; the autotuner's cache works; the HBM
budget is enforced."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2511_02328_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5

BEAMS = [
    # nchan, f_lo, f_hi, tsamp, nsamp, dms, widths, thresh
    (96, 1000.0, 1500.0, 2e-4, 12000, np.arange(0, 60, 1.0), [1, 2, 4, 8], 7.0),
    (256, 1100.0, 1400.0, 1e-4, 20000, np.arange(0, 30, 0.5), [1, 4, 16], 6.0),
    (33, 1500.0, 1000.0, 5e-4, 5003, np.arange(0, 100, 2.0), [1, 2, 3], 6.5),
    (512, 1000.0, 1500.0, 1e-4, 16384, np.arange(0, 25, 1.0), [1, 2, 4, 8, 16, 32], 7.0),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _make(seed, with_pulses=True):
    data = []
    for i, (nchan, f_lo, f_hi, tsamp, nsamp, dms, widths, thr) in enumerate(BEAMS):
        pulses = []
        if with_pulses:
            offs = oracle.injection_offsets(nchan, f_lo, f_hi, tsamp, float(dms[len(dms) // 2]), nsamp // 3)
            pulses = [synth.Pulse(offs, 3, synth.pulse_amplitude(25.0, nchan, 3))]
        x = synth.filterbank(nchan, nsamp, seed=seed * 100 + i, pulses=pulses)
        data.append(x)
    return data


def _build(xs_dev, budget=0):
    from paper_2511_02328_gb300 import _lib
    descs = []
    for (nchan, f_lo, f_hi, tsamp, nsamp, dms, widths, thr), xd in zip(BEAMS, xs_dev):
        descs.append(dict(nchan=nchan, f_lo=f_lo, f_hi=f_hi, tsamp=tsamp, dm_list=dms, d_in=xd.data_ptr(),
                          nsamp=nsamp, widths=widths, thresh=thr, cap=1 << 14))
    return _lib.af_batch_build(descs, budget)


def _check_against_oracle(batch, xs):
    from paper_2511_02328_gb300 import _lib
    for i, ((nchan, f_lo, f_hi, tsamp, nsamp, dms, widths, thr), x) in enumerate(zip(BEAMS, xs)):
        from paper_2511_02328_gb300.search import device_view
        pl, sn, bw, nout = _lib.af_batch_buffers(batch, i)
        plane = device_view(pl, (len(dms), nout), torch.int32)
        snr = device_view(sn, (len(dms), nout), torch.float32)
        D = oracle.delay_table(nchan, f_lo, f_hi, tsamp, dms)
        Y = oracle.dedisperse(x, D)
        assert np.array_equal(plane.cpu().numpy(), Y), "beam %d plane" % i
        ref, _ = oracle.boxcar_snr(Y, widths)
        got = snr.cpu().numpy().astype(np.float64)
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(got), fin)
        err = np.abs(got[fin] - ref[fin]) / np.maximum(1.0, np.abs(ref[fin]))
        assert float(err.max()) <= TOL, (i, float(err.max()))


@pytest.mark.parametrize("strategy", ["auto", "tile", "pairs", "persistent"])
def test_batch_matches_oracle_and_single_beam(strategy, monkeypatch):
    """Every dedispersion strategy of the batch (the autotuner's pick, the
    persistent tile kernel, group rows beam after beam, persistent group rows
    over all beams in waves) gives each beam's oracle plane and S/N and the
    single-beam host search's candidates."""
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import Plan
    if strategy != "auto":
        monkeypatch.setenv("AFGB_BATCH_STRATEGY", strategy)
    if strategy in ("pairs", "persistent"):
        monkeypatch.setenv("AFGB_DEDISP_KERNEL", "pairs")   # every beam that can, on group rows
    xs = _make(1)
    xs_dev = [torch.from_numpy(x).cuda() for x in xs]
    batch = _build(xs_dev)
    nw, m, ms, cached = _lib.af_batch_shape(batch)
    if strategy == "persistent" or (strategy == "auto" and m < 0):
        assert nw in (2, 3, 4) and m < 0           # ring depth, -(tiles per wave)
    else:
        assert (nw, m) in {"auto": [(11, 8), (7, 8), (15, 6), (15, 0)], "tile": [(11, 8), (7, 8), (15, 6)],
                           "pairs": [(15, 0)]}[strategy]
    tuning = _lib.af_batch_tuning(batch)
    assert len(tuning) >= 1 and all(t["ms"] > 0 for t in tuning)
    if strategy == "auto":                          # every kind of strategy was timed
        assert {t["kind"] for t in tuning} == {0, 1, 2}
    _lib.af_batch_run(batch, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    _check_against_oracle(batch, xs)
    for i, ((nchan, f_lo, f_hi, tsamp, nsamp, dms, widths, thr), x) in enumerate(zip(BEAMS, xs)):
        got, n = _lib.af_batch_candidates(batch, i, 1 << 14)
        p = Plan(nchan, f_lo, f_hi, tsamp, dms)
        ref, nref = p.search_host(x, widths, thr, cap=1 << 14)
        assert n == nref and np.array_equal(got, ref), i
        assert n >= 1
        p.close()
    _lib.af_batch_destroy(batch)


def test_graph_replay_sees_new_input():
    from paper_2511_02328_gb300 import _lib
    xs = _make(2)
    xs_dev = [torch.from_numpy(x).cuda() for x in xs]
    batch = _build(xs_dev)
    s = torch.cuda.Stream()
    _lib.af_batch_run(batch, s.cuda_stream)
    s.synchronize()
    first = [_lib.af_batch_candidates(batch, i, 1 << 14) for i in range(len(BEAMS))]
    # replay on the same data: identical
    _lib.af_batch_run(batch, s.cuda_stream)
    s.synchronize()
    again = [_lib.af_batch_candidates(batch, i, 1 << 14) for i in range(len(BEAMS))]
    for (a, na), (b, nb) in zip(first, again):
        assert na == nb and np.array_equal(a, b)
    # new data in the same buffers: the replayed graph computes on it
    ys = _make(3, with_pulses=False)
    for xd, y in zip(xs_dev, ys):
        xd.copy_(torch.from_numpy(y))
    torch.cuda.synchronize()
    _lib.af_batch_run(batch, s.cuda_stream)
    s.synchronize()
    _check_against_oracle(batch, ys)
    _lib.af_batch_destroy(batch)


def test_autotune_cache(tmp_path, monkeypatch):
    from paper_2511_02328_gb300 import _lib
    path = tmp_path / "tune.json"
    monkeypatch.setenv("AFGB_AUTOTUNE_CACHE", str(path))
    xs_dev = [torch.from_numpy(x).cuda() for x in _make(4, with_pulses=False)]
    b1 = _build(xs_dev)
    nw, m, ms, cached = _lib.af_batch_shape(b1)
    assert not cached and ms > 0
    doc = json.loads(path.read_text())
    assert len(doc) == 1
    entry = list(doc.values())[0]
    assert (entry["nw"], entry["m"]) == (nw, m)
    b2 = _build(xs_dev)
    nw2, m2, _, cached2 = _lib.af_batch_shape(b2)
    assert cached2 and (nw2, m2) == (nw, m)
    _lib.af_batch_destroy(b1)
    _lib.af_batch_destroy(b2)


def test_hbm_budget_rejected():
    from paper_2511_02328_gb300 import _lib
    xs_dev = [torch.from_numpy(x).cuda() for x in _make(5, with_pulses=False)]
    with pytest.raises(_lib.AFError) as e:
        _build(xs_dev, budget=1 << 20)
    assert e.value.code == _lib.AF_ENOBUFS


def test_full_multibeam_batch_sampled_rows():
    # The full 19-beam workload of the bench (10.7 GB of input, nchan 1024-4096,
    # DM up to 2000, 2^16-2^19 samples) in one batch: two sampled rows of every
    # beam are bit-exact with the oracle, their S/N within tolerance, and the
    # batch's candidate counts equal the per-plan path's on two beams.
    from paper_2511_02328_gb300 import _lib, workloads
    from paper_2511_02328_gb300.search import Plan, device_view

    def dmax_of(nchan, f_lo, f_hi, tsamp, dm):
        return int(oracle.delay_table(nchan, f_lo, f_hi, tsamp, [dm]).max())

    beams = workloads.multibeam(19, dmax_of)
    xs, descs = [], []
    for b, bm in enumerate(beams):
        xs.append(synth.filterbank_torch(bm["nchan"], bm["nsamp"], seed=700 + b, device="cuda"))
        descs.append(dict(nchan=bm["nchan"], f_lo=bm["f_lo"], f_hi=bm["f_hi"], tsamp=bm["tsamp"],
                          dm_list=bm["dm_list"], d_in=xs[-1].data_ptr(), nsamp=bm["nsamp"], widths=bm["widths"],
                          thresh=bm["thresh"], cap=1 << 16))
    batch = _lib.af_batch_build(descs)
    _lib.af_batch_run(batch, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for i, bm in enumerate(beams):
        pl, sn, _, nout = _lib.af_batch_buffers(batch, i)
        ndm = len(bm["dm_list"])
        rows = [0, ndm - 1] if i % 2 else [ndm // 3, (2 * ndm) // 3]
        plane = device_view(pl, (ndm, nout), torch.int32)
        snr = device_view(sn, (ndm, nout), torch.float32)
        x = xs[i].cpu().numpy()
        D = oracle.delay_table(bm["nchan"], bm["f_lo"], bm["f_hi"], bm["tsamp"], bm["dm_list"])
        Y = oracle.dedisperse(x, D[rows], nout)
        assert np.array_equal(plane[rows].cpu().numpy(), Y), i
        ref, _ = oracle.boxcar_snr(Y, bm["widths"])
        got = snr[rows].cpu().numpy().astype(np.float64)
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(got), fin)
        assert float((np.abs(got[fin] - ref[fin]) / np.maximum(1.0, np.abs(ref[fin]))).max()) <= TOL, i
        if i in (0, 11):
            _, n = _lib.af_batch_candidates(batch, i, 1 << 16)
            p = Plan(bm["nchan"], bm["f_lo"], bm["f_hi"], bm["tsamp"], bm["dm_list"])
            _, nref = p.search_host(x, bm["widths"], bm["thresh"], cap=1 << 16)
            assert n == nref, i
            p.close()
    _lib.af_batch_destroy(batch)
