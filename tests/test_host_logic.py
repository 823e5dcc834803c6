"""Host logic that needs no GPU: the classifier's true-positive matching
(Sec. 4.2) and its equal-recall comparison, and the benchmark's summary of the
clock samples.  The matching is pinned against the oracle's independent
restatement of the rule; the rest against cases worked out by hand."""
import numpy as np
import pytest

from paper_2511_02328_gb300 import _lib, classifier
import bench
from oracle import nms


def _reps(rows):
    """rows: (dm_idx, abs_sample, snr) -> candidate records as the search returns them."""
    a = np.zeros(len(rows), dtype=_lib.CAND_DTYPE)
    for i, (d, s, snr) in enumerate(rows):
        a[i]["dm_idx"], a[i]["t"], a[i]["abs_sample"], a[i]["snr"], a[i]["width"] = d, s, s, snr, 1
    return a


def test_match_tolerances_are_strict():
    # Sec. 4.2: a true positive needs |dDM| < 20 and |dTOA| < 0.2 s (both strict).
    dms = np.arange(0.0, 501.0)
    tsamp = 1e-3
    reps = _reps([(100, 1000, 9.0)])                      # DM 100, TOA 1.0 s
    assert classifier.match(reps, [(119.5, 1.15, 10, 9.0)], dms, tsamp)[0] == 0
    assert classifier.match(reps, [(80.5, 0.85, 10, 9.0)], dms, tsamp)[0] == 0
    assert classifier.match(reps, [(120.0, 1.0, 10, 9.0)], dms, tsamp)[0] == -1    # |dDM| = 20
    assert classifier.match(reps, [(80.0, 1.0, 10, 9.0)], dms, tsamp)[0] == -1
    assert classifier.match(reps, [(100.0, 1.25, 10, 9.0)], dms, tsamp)[0] == -1   # |dTOA| > 0.2 s
    assert classifier.match(reps, [(100.0, 0.75, 10, 9.0)], dms, tsamp)[0] == -1
    # the first injection within both tolerances is the one reported
    inj = [(300.0, 1.0, 10, 9.0), (105.0, 1.1, 10, 9.0), (95.0, 0.95, 10, 9.0)]
    assert classifier.match(reps, inj, dms, tsamp)[0] == 1
    assert len(classifier.match(_reps([]), inj, dms, tsamp)) == 0


def test_match_agrees_with_the_oracle_rule():
    # With injections more than 2 x 0.2 s apart each cluster can match at most one,
    # so the per-cluster indices give exactly the oracle's recalled set and FP count.
    rng = np.random.default_rng(7)
    dms = np.arange(0.0, 501.0)
    tsamp = 98.304e-6
    for _ in range(20):
        ninj = int(rng.integers(0, 6))
        toas = 0.5 + 0.45 * np.arange(ninj) + rng.uniform(0.0, 0.02, ninj)
        inj = [(float(rng.uniform(20, 480)), float(t), 10, float(rng.uniform(6, 30))) for t in toas]
        rows = []
        for _ in range(int(rng.integers(0, 12))):
            if inj and rng.random() < 0.6:
                idm, itoa = inj[int(rng.integers(0, ninj))][:2]
                d = int(np.clip(round(idm + rng.uniform(-30, 30)), 0, 500))
                s = int(round((itoa + rng.uniform(-0.3, 0.3)) / tsamp))
            else:
                d, s = int(rng.integers(0, 501)), int(rng.integers(0, 30000))
            rows.append((d, max(s, 0), float(rng.uniform(6, 20))))
        reps = _reps(rows)
        got = classifier.match(reps, inj, dms, tsamp)
        hit, fp = nms.match([(int(r["dm_idx"]), int(r["abs_sample"])) for r in reps],
                            [(i[0], i[1]) for i in inj], dms, tsamp)
        assert int((got < 0).sum()) == fp
        assert set(int(j) for j in got if j >= 0) == {j for j, h in enumerate(hit) if h}


def _records():
    """Three chunks, worked by hand.  Injections are (dm, toa, width, S/N);
    clusters are (S/N, index of the injection matched or -1)."""
    chunk0 = dict(snr=np.array([10.0, 7.0, 9.0]), match=np.array([0, 1, -1]),
                  inj=[(100.0, 1.0, 10, 12.0), (200.0, 2.0, 10, 9.0), (300.0, 3.0, 10, 5.0)], start=0, n=3)
    chunk1 = dict(snr=np.array([8.2, 20.0]), match=np.array([0, -1]),
                  inj=[(50.0, 0.5, 10, 8.5)], start=3, n=2)
    chunk2 = dict(snr=np.zeros(0), match=np.zeros(0, dtype=np.int64), inj=[(70.0, 0.7, 10, 30.0)], start=5, n=0)
    return [chunk0, chunk1, chunk2]


def test_equal_recall_on_a_worked_example():
    recs = _records()
    snr = np.concatenate([r["snr"] for r in recs])
    prob = np.array([0.9, 0.8, 0.1, 0.7, 0.2])
    res = classifier.evaluate(snr, prob, recs, thresh=8.0, min_inj_snr=8.0, tsamp=1e-3, nout=1000)
    # injections with S/N >= 8: chunk 0's first two, chunk 1's, chunk 2's (no cluster): 4
    assert res["injected"] == 4
    # S/N >= 8 keeps clusters 0, 2 (chunk 0) and both of chunk 1: injections 0/0 and 1/0 found;
    # cluster 2 of chunk 0 and cluster 1 of chunk 1 match nothing
    assert res["recall_threshold"] == pytest.approx(2 / 4)
    assert res["fp_threshold"] == 2
    # S/N >= 6 and P >= p: p = 0.9 finds one injection (1/4 < 2/4 - 1 %); p = 0.8 adds the S/N-7
    # cluster of injection 0/1, reaching 2/4 with no false positive
    assert res["p_cut"] == pytest.approx(0.8)
    assert res["recall_cnn"] == pytest.approx(2 / 4)
    assert res["fp_cnn"] == 0
    # three chunks of 1000 samples of 1 ms
    assert res["hours"] == pytest.approx(3.0 / 3600.0)
    assert res["fp_per_hour_threshold"] == pytest.approx(2 / (3.0 / 3600.0))


def test_equal_recall_takes_the_highest_cut_within_one_percent():
    # 250 chunks with one injection each: the threshold finds 125 of them (S/N-9 clusters),
    # the other 125 have S/N-7 clusters.  Probabilities fall with the chunk index, so the
    # cut p admits the first k clusters; recall k/250 reaches 0.5 - 0.01 first at k = 123
    # (122/250 = 0.488 falls short), which fixes p at the 123rd probability.
    recs, snr, prob = [], [], []
    for k in range(250):
        s = 9.0 if k < 125 else 7.0
        recs.append(dict(snr=np.array([s]), match=np.array([0]), inj=[(100.0, 1.0, 10, 12.0)], start=k, n=1))
        snr.append(s)
        prob.append(1.0 - k / 1000.0)
    res = classifier.evaluate(np.array(snr), np.array(prob), recs, nout=1000, tsamp=1e-3)
    assert res["recall_threshold"] == pytest.approx(0.5)
    assert res["recall_cnn"] == pytest.approx(123 / 250)
    assert res["p_cut"] == pytest.approx(1.0 - 122 / 1000.0)
    assert res["fp_cnn"] == 0 and res["fp_threshold"] == 0


def test_clock_summary():
    s = bench.ClockSampler(0)
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    s.rows = [
        ["2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["1980", "2070", "1390.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
        ["[N/A]", "2070", "1", "0x0", "Active", "Active", "Active", "Active"],   # unparsable: skipped
        ["2040", "2070", "1200.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
    ]
    out = s.summary()
    assert out["sm_mhz"] == 2040.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    s.rows.append(["1500", "2070", "1400", "0x8", "Active", "Not Active", "Active", "Not Active"])
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
