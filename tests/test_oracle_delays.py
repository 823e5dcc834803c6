"""Pins for the oracle's delay table (Eq. KDM, Eq. coarse_delay, Sec. 2.3)."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from conftest import C1, C2, dm_list

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_physical_delay_dm1000():
    # Closed form: K * 1000 * (1/1000^2 - 1/1500^2) = 4148.808 * 5/9 * 1e-3 s.
    # With K in seconds this is the textbook 2.305 s; with the printed "ms" it
    # would be 2.3 ms, which is not physical.
    fr = 1500.0
    tsamp = 1e-6
    n, x = brute.exact_delay(1000.0, 1000.0, fr, tsamp)
    assert abs(float(x) * tsamp - 4148.808 * 5.0 / 9.0 * 1e-3) < 1e-12
    assert abs(float(x) * tsamp - 2.304893) < 1e-6


def test_channel_centres_and_reference():
    f = oracle.chan_freqs(4, 1000.0, 1400.0)
    assert np.allclose(f, [1050.0, 1150.0, 1250.0, 1350.0])
    f = oracle.chan_freqs(4, 1400.0, 1000.0)
    assert np.allclose(f, [1350.0, 1250.0, 1150.0, 1050.0])
    assert oracle.lib().oracle_ref_freq(1000.0, 1500.0) == 1500.0
    assert oracle.lib().oracle_ref_freq(1500.0, 1000.0) == 1500.0


@pytest.mark.parametrize("cfg", [C1, C2], ids=["c1", "c2"])
def test_delays_match_exact_rational(cfg):
    dms = dm_list(cfg)
    D = oracle.delay_table(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms)
    rng = np.random.default_rng(7)
    fr = max(cfg["f_lo"], cfg["f_hi"])
    df = (cfg["f_hi"] - cfg["f_lo"]) / cfg["nchan"]
    idx = list(zip(rng.integers(0, len(dms), 400), rng.integers(0, cfg["nchan"], 400)))
    idx += [(len(dms) - 1, 0), (len(dms) - 1, cfg["nchan"] - 1), (1, 0)]
    for d, c in idx:
        fc = cfg["f_lo"] + (c + 0.5) * df
        n, x = brute.exact_delay(dms[d], fc, fr, cfg["tsamp"])
        # a tie within double rounding would make the comparison ambiguous
        assert abs(abs(x - int(x)) - 0.5) > 1e-9
        assert D[d, c] == n, (d, c, D[d, c], n, float(x))


@pytest.mark.parametrize("cfg", [C1, C2, dict(C2, dm_hi=2000.0)], ids=["c1", "c2", "stream"])
def test_no_rounding_ties_in_the_workload_tables(cfg):
    # Rounding reading: half away from zero.  On the workloads' whole tables no
    # product a*b (Eq. coarse_delay, same operation order in IEEE double) lies
    # within 1e-9 of a .5 tie, so round-half-to-even gives the same table and
    # the tie rule never decides a delay here.
    dms = dm_list(cfg)
    D = oracle.delay_table(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms)
    K = float(json.load(open(os.path.join(GOLDEN, "paper_constants.json")))["K_DM"]["value"])
    df = (cfg["f_hi"] - cfg["f_lo"]) / cfg["nchan"]
    fc = cfg["f_lo"] + (np.arange(cfg["nchan"], dtype=np.float64) + 0.5) * df
    fr = max(cfg["f_lo"], cfg["f_hi"])
    a = (K * dms) / cfg["tsamp"]
    b = 1.0 / (fc * fc) - 1.0 / (fr * fr)
    x = a[:, None] * b[None, :]
    frac = x - np.floor(x)
    assert int(np.count_nonzero(np.abs(frac - 0.5) < 1e-9)) == 0
    assert np.array_equal(np.rint(x).astype(np.int64), D.astype(np.int64))


def test_dmax_closed_form():
    # Dmax = delay of the lowest channel centre at the largest DM.
    for cfg, expect in [(C1, 11682), (C2, 46883)]:
        dms = dm_list(cfg)
        D = oracle.delay_table(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms)
        fc0 = cfg["f_lo"] + 0.5 * (cfg["f_hi"] - cfg["f_lo"]) / cfg["nchan"]
        n, _ = brute.exact_delay(dms[-1], fc0, cfg["f_hi"], cfg["tsamp"])
        assert int(D.max()) == n == expect
        assert oracle.lib().oracle_dmax(D.ctypes.data, D.shape[0], D.shape[1]) == expect


def test_delay_invariants():
    cfg = C1
    dms = dm_list(cfg)
    D = oracle.delay_table(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms)
    assert np.all(D[0] == 0)                       # DM 0: no delay
    assert np.all(np.diff(D, axis=0) >= 0)         # monotone in DM per channel
    assert np.all(np.diff(D, axis=1) <= 0)         # lower frequency (small c) arrives later
    assert np.all(D >= 0)
    # top channel centre is half a channel (df/2) below f_ref: to first order the
    # delay is 2 K DM (df/2) / f^3 / tsamp, about 12 samples at DM 500
    df = (cfg["f_hi"] - cfg["f_lo"]) / cfg["nchan"]
    approx = 2 * 4148.808 * dms[-1] * (df / 2) / cfg["f_hi"] ** 3 / cfg["tsamp"]
    assert abs(D[-1, -1] - approx) <= 1.0 and D[-1, -1] > 0


def test_descending_band_is_reversed():
    dms = np.array([0.0, 3.5, 100.0, 777.0])
    A = oracle.delay_table(64, 1000.0, 1500.0, 64e-6, dms)
    B = oracle.delay_table(64, 1500.0, 1000.0, 64e-6, dms)
    assert np.array_equal(A[:, ::-1], B)


def test_non_monotone_dm_list_is_per_row():
    dms = np.array([300.0, 0.0, 12.25, 299.0])
    A = oracle.delay_table(32, 1000.0, 1500.0, 1e-4, dms)
    for i, dm in enumerate(dms):
        assert np.array_equal(A[i], oracle.delay_table(32, 1000.0, 1500.0, 1e-4, [dm])[0])


def test_invalid_arguments():
    with pytest.raises(ValueError):
        oracle.delay_table(8, 1000.0, 1000.0, 1e-4, [1.0])
    with pytest.raises(ValueError):
        oracle.delay_table(8, 1000.0, 1500.0, 1e-4, [-1.0])
    with pytest.raises(ValueError):
        oracle.delay_table(8, 1000.0, 1500.0, 0.0, [1.0])
