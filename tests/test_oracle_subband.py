"""Pins for the oracle's two-stage subband dedispersion (Sec. 2.3, Eqs. stage1,
residual, stage2, sb_smear).

Each test checks the oracle against something other than its own formula:
numpy's median, the closed form of the 1/f^2-weighted centre, exact rational
arithmetic, the brute-force oracle (N0 = 1, one subband, the effective-delay
regrouping of the double sum), a pure-Python loop restatement on tiny inputs,
and the smearing estimate of Eq. (sb_smear).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import brute
from conftest import C1, dm_list

K = 4.148808e3


def _centres(nchan, f_lo, f_hi):
    return oracle.chan_freqs(nchan, f_lo, f_hi)


@pytest.mark.parametrize("nchan,nsub", [(256, 16), (48, 5), (7, 7), (4096, 64), (255, 17), (10, 1)])
def test_partition_invariants(nchan, nsub):
    first = oracle.subband_first(nchan, nsub)
    assert first[0] == 0 and first[-1] == nchan
    sizes = np.diff(first)
    assert np.all(sizes >= 1)
    assert sizes.max() - sizes.min() <= 1
    assert sizes.sum() == nchan


def test_partition_reading_example():
    # Reading: subband s starts at floor(s * nchan / nsub), so the larger
    # subbands come last.
    assert oracle.subband_first(10, 4).tolist() == [0, 2, 5, 7, 10]
    assert oracle.subband_first(4096, 64).tolist() == list(range(0, 4097, 64))


def test_partition_rejects_more_subbands_than_channels():
    with pytest.raises(ValueError):
        oracle.subband_first(4, 5)


@pytest.mark.parametrize("nchan,nsub,f_lo,f_hi", [(256, 16, 1000.0, 1500.0), (48, 5, 1500.0, 1000.0),
                                                   (30, 4, 1200.0, 1450.0), (9, 9, 1000.0, 1500.0)])
def test_median_frequency_is_numpy_median(nchan, nsub, f_lo, f_hi):
    f = _centres(nchan, f_lo, f_hi)
    first = oracle.subband_first(nchan, nsub)
    F = oracle.subband_freqs(nchan, f_lo, f_hi, nsub, oracle.FS_MEDIAN)
    for s in range(nsub):
        assert F[s] == pytest.approx(np.median(f[first[s]:first[s + 1]]), rel=1e-15, abs=0)


@pytest.mark.parametrize("nchan,nsub,f_lo,f_hi", [(256, 16, 1000.0, 1500.0), (48, 5, 1500.0, 1000.0),
                                                   (9, 9, 1000.0, 1500.0)])
def test_invsq_frequency_closed_form(nchan, nsub, f_lo, f_hi):
    # 1/F^2 is the mean of 1/f^2 over the subband; F lies inside the subband,
    # below its median (1/f^2 is convex); a one-channel subband gives f_c.
    f = _centres(nchan, f_lo, f_hi)
    first = oracle.subband_first(nchan, nsub)
    F = oracle.subband_freqs(nchan, f_lo, f_hi, nsub, oracle.FS_INVSQ)
    for s in range(nsub):
        fs = f[first[s]:first[s + 1]]
        assert 1.0 / F[s] ** 2 == pytest.approx(np.mean(1.0 / fs ** 2), rel=1e-14)
        assert fs.min() <= F[s] <= fs.max()
        assert F[s] <= np.median(fs) * (1 + 1e-15)
        if fs.size == 1:
            assert F[s] == pytest.approx(fs[0], rel=1e-15)


@pytest.mark.parametrize("mode", [oracle.FS_MEDIAN, oracle.FS_INVSQ])
def test_residual_shifts_exact_rational(mode):
    cfg = C1
    nchan, nsub, n0 = cfg["nchan"], 16, 8
    dms = dm_list(cfg)
    tab = oracle.subband_tables(nchan, cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms, n0, nsub, mode)
    f = _centres(nchan, cfg["f_lo"], cfg["f_hi"])
    first = tab["first"]
    fr = max(cfg["f_lo"], cfg["f_hi"])
    ties = 0
    for s in range(nsub):
        fs = [Fraction(float(x)) for x in f[first[s]:first[s + 1]]]
        if mode == oracle.FS_MEDIAN:
            inv_f2 = 1 / Fraction(float(np.median(f[first[s]:first[s + 1]]))) ** 2
        else:
            inv_f2 = sum(1 / x ** 2 for x in fs) / len(fs)
        for m in range(0, len(dms), 3):
            ddm = dms[m] - dms[(m // n0) * n0]
            n, x = brute.exact_shift(ddm, inv_f2, fr, cfg["tsamp"])
            if abs(abs(x - int(x)) - Fraction(1, 2)) < Fraction(1, 10 ** 6):
                ties += 1
                continue
            assert tab["R"][m, s] == n, (m, s, tab["R"][m, s], float(x))
    assert ties <= 2
    # the first DM of every group is on the coarse grid: no residual
    assert np.all(tab["R"][::n0] == 0)
    assert np.all(tab["R"] >= 0)


def test_coarse_delays_are_the_plain_delay_table():
    cfg = C1
    dms = dm_list(cfg)
    tab = oracle.subband_tables(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms, 8, 16, oracle.FS_MEDIAN)
    D = oracle.delay_table(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms)
    assert np.array_equal(tab["Dc"], D[::8])
    assert tab["Dc"].shape[0] == (len(dms) + 7) // 8


def _random_case(seed, nchan, nsamp, f_lo, f_hi, tsamp, dms, n0, nsub, mode):
    rng = np.random.default_rng(seed)
    X = rng.integers(0, 256, size=(nchan, nsamp), dtype=np.uint8)
    tab = oracle.subband_tables(nchan, f_lo, f_hi, tsamp, dms, n0, nsub, mode)
    return X, tab


CASES = [
    # seed, nchan, nsamp, f_lo, f_hi, tsamp, dms, n0, nsub, mode
    (1, 48, 3000, 1000.0, 1500.0, 98.304e-6, np.arange(0.0, 40.0, 0.7), 4, 5, oracle.FS_MEDIAN),
    (2, 64, 4096, 1500.0, 1000.0, 98.304e-6, np.arange(3.0, 60.0, 1.0), 8, 8, oracle.FS_INVSQ),
    (3, 33, 2500, 1200.0, 1450.0, 65.536e-6, np.array([0.0, 0.0, 1.0, 5.0, 5.5, 9.0, 30.0]), 3, 4, oracle.FS_INVSQ),
    (4, 16, 1500, 1000.0, 1500.0, 98.304e-6, np.arange(0.0, 20.0, 1.0), 5, 16, oracle.FS_MEDIAN),
]


@pytest.mark.parametrize("case", CASES, ids=[str(c[0]) for c in CASES])
def test_plane_is_brute_force_with_effective_delays(case):
    # Regrouping the double sum of Eqs. (stage1)-(stage2): every channel c of
    # subband s is read at v + R[m][s] + D[j(m)][c].  The brute-force oracle with
    # that table is an independent code path.
    X, tab = _random_case(*case)
    Deff = oracle.subband_effective_delays(tab)
    Y = oracle.subband_dedisperse(X, tab)
    assert Y.shape[1] == X.shape[1] - int(Deff.max())
    assert np.array_equal(Y, oracle.dedisperse(X, Deff, Y.shape[1]))


@pytest.mark.parametrize("nsub", [1, 7, 64])
def test_n0_one_is_the_brute_force_plane(nsub):
    # N0 = 1: every fine DM is on the coarse grid, the residuals vanish and the
    # two stages reduce to the brute-force sum (Sec. 2.3).
    rng = np.random.default_rng(11)
    nchan, nsamp = 64, 4000
    dms = np.arange(0.0, 50.0, 1.5)
    X = rng.integers(0, 256, size=(nchan, nsamp), dtype=np.uint8)
    tab = oracle.subband_tables(nchan, 1000.0, 1500.0, 98.304e-6, dms, 1, nsub, oracle.FS_MEDIAN)
    assert np.all(tab["R"] == 0)
    D = oracle.delay_table(nchan, 1000.0, 1500.0, 98.304e-6, dms)
    Y = oracle.subband_dedisperse(X, tab)
    assert np.array_equal(Y, oracle.dedisperse(X, D))


def test_single_subband_is_shifted_coarse_plane():
    # One subband: Y(m, v) = I(j, 0, v + R_m) = the brute-force plane of the
    # coarse DM j, shifted by the residual R_m.
    rng = np.random.default_rng(5)
    nchan, nsamp, n0 = 40, 5000, 6
    dms = np.arange(0.0, 45.0, 1.0)
    X = rng.integers(0, 256, size=(nchan, nsamp), dtype=np.uint8)
    tab = oracle.subband_tables(nchan, 1000.0, 1500.0, 98.304e-6, dms, n0, 1, oracle.FS_INVSQ)
    Y = oracle.subband_dedisperse(X, tab)
    nout = Y.shape[1]
    for m in range(len(dms)):
        j, r = m // n0, int(tab["R"][m, 0])
        Yc = oracle.dedisperse(X, tab["Dc"][j:j + 1], nsamp - int(tab["Dc"][j].max()))[0]
        assert np.array_equal(Y[m], Yc[r:r + nout]), m


@pytest.mark.parametrize("case", [
    (7, 6, 60, 1000.0, 1500.0, 98.304e-6, np.arange(0.0, 1.6, 0.2), 3, 2, oracle.FS_MEDIAN),
    (8, 5, 50, 1500.0, 1100.0, 98.304e-6, np.array([0.0, 0.5, 0.5, 1.25, 2.0]), 2, 3, oracle.FS_INVSQ),
])
def test_tiny_two_stage_loops(case):
    X, tab = _random_case(*case)
    Y = oracle.subband_dedisperse(X, tab)
    Yb = brute.subband_dedisperse(X.tolist(), tab["Dc"].tolist(), tab["first"].tolist(), tab["R"].tolist(),
                                  tab["n0"], Y.shape[1])
    assert Y.tolist() == Yb


def _smearing(tab, cfg, dms):
    """Deviation of the effective delay from the exact fine-DM delay, and the
    first-order smearing of Eq. (sb_smear) per (m, c), both in samples."""
    nchan = tab["nchan"]
    f = _centres(nchan, cfg["f_lo"], cfg["f_hi"])
    fr = max(cfg["f_lo"], cfg["f_hi"])
    Deff = oracle.subband_effective_delays(tab).astype(np.float64)
    exact = K * dms[:, None] / cfg["tsamp"] * (1.0 / f[None, :] ** 2 - 1.0 / fr ** 2)
    sub_of = np.repeat(np.arange(tab["nsub"]), np.diff(tab["first"]))
    F = tab["F"][sub_of]
    ddm = dms - dms[(np.arange(len(dms)) // tab["n0"]) * tab["n0"]]
    width = np.abs(f[1] - f[0]) * np.diff(tab["first"])[sub_of]          # subband width Delta f_s
    smear = 2.0 * K * ddm[:, None] * width[None, :] / F[None, :] ** 3 / cfg["tsamp"]
    return Deff - exact, smear, width / F


def test_smearing_bound_median_centre():
    # Eq. (sb_smear): with F_s at the subband centre every channel is within
    # Delta f_s / 2 of it, so the effective delay is within one sample (two
    # roundings) plus half the first-order smearing (and a second-order margin)
    # of the exact fine-DM delay; the extreme channels reach that half.
    cfg = C1
    dms = dm_list(cfg)
    tab = oracle.subband_tables(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms, 16, 16, oracle.FS_MEDIAN)
    dev, smear, rel = _smearing(tab, cfg, dms)
    half = 0.5 * smear * (1.0 + 2.0 * rel[None, :])
    assert np.all(np.abs(dev) <= 1.0 + half + 1e-9)
    big = smear > 10
    assert big.any()
    assert np.max(np.abs(dev[big]) / (0.5 * smear[big])) > 0.8


def test_smearing_invsq_centre_is_unbiased():
    # With 1/F_s^2 = mean 1/f_c^2 the residual error K*dDM*(1/F_s^2 - 1/f_c^2)
    # averages to zero over each subband, so the mean deviation per (m, s) is
    # rounding only; the median centre leaves a bias that grows with dDM.
    cfg = C1
    dms = dm_list(cfg)
    for mode, biased in [(oracle.FS_INVSQ, False), (oracle.FS_MEDIAN, True)]:
        tab = oracle.subband_tables(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms, 16, 2, mode)
        dev, smear, _ = _smearing(tab, cfg, dms)
        first = tab["first"]
        means = np.stack([dev[:, first[s]:first[s + 1]].mean(axis=1) for s in range(tab["nsub"])], axis=1)
        if biased:
            assert np.max(np.abs(means)) > 1.5
        else:
            assert np.max(np.abs(means)) <= 1.0 + 1e-9
        assert np.all(np.abs(dev) <= 1.0 + smear * 1.05 + 1e-9)


def test_injected_pulse_snr_loss_is_small():
    # A pulse between coarse DMs: the subband plane keeps most of the
    # brute-force S/N when the smearing is below the pulse width (measured,
    # not a bound: the paper quotes no S/N loss).
    from paper_2511_02328_gb300 import synth
    cfg = C1
    dms = dm_list(cfg)
    nchan, nsamp = cfg["nchan"], cfg["nsamp"]
    dm0, t0, w = 301.0, 9000, 10            # DM 301 lies between coarse DMs 296 and 304
    offs = oracle.injection_offsets(nchan, cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dm0, t0)
    amp = synth.pulse_amplitude(15.0, nchan, w)
    X = synth.filterbank(nchan, nsamp, seed=3, pulses=[synth.Pulse(offs, w, amp)])
    tab = oracle.subband_tables(nchan, cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms, 8, 32, oracle.FS_INVSQ)
    Ys = oracle.subband_dedisperse(X, tab)
    D = oracle.delay_table(nchan, cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms)
    Yb = oracle.dedisperse(X, D)
    rows = slice(290, 312)
    ss, _ = oracle.boxcar_snr(Ys[rows], [8, 16])
    sb, _ = oracle.boxcar_snr(Yb[rows], [8, 16])
    best_s, best_b = ss.max(), sb.max()
    assert best_b > 12
    assert best_s > 0.9 * best_b
    # the peak stays at the injected DM within the smearing
    d_s = np.unravel_index(np.argmax(ss), ss.shape)[0] + 290
    assert abs(dms[d_s] - dm0) <= 3
