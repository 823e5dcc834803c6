"""Pins for the oracle's zero-DM filter and robust (median/MAD) S/N
normalisation (Sec. 2.1 RFI mitigation, Sec. 4.4)."""
import numpy as np
import pytest

import oracle
from paper_2511_02328_gb300 import synth


def _zerodm_loops(X):
    nchan, nsamp = len(X), len(X[0])
    out = [[0] * nsamp for _ in range(nchan)]
    for t in range(nsamp):
        s = sum(int(X[c][t]) for c in range(nchan))
        # mean rounded half up, by counting: the largest q with q <= s/nchan + 1/2
        q = 0
        while 2 * (q + 1) * nchan <= 2 * s + nchan:
            q += 1
        for c in range(nchan):
            out[c][t] = min(255, max(0, int(X[c][t]) - q + 128))
    return out


def test_zerodm_tiny_loops():
    rng = np.random.default_rng(2)
    for nchan, nsamp in [(1, 5), (2, 7), (5, 9), (16, 13)]:
        X = rng.integers(0, 256, size=(nchan, nsamp), dtype=np.uint8)
        assert oracle.zerodm(X).tolist() == _zerodm_loops(X.tolist())


def test_zerodm_half_rounds_up():
    X = np.array([[1], [2]], dtype=np.uint8)           # mean 1.5 -> 2
    assert oracle.zerodm(X)[:, 0].tolist() == [127, 128]
    X = np.array([[1], [2], [2], [2]], dtype=np.uint8)  # mean 1.75 -> 2
    assert oracle.zerodm(X)[:, 0].tolist() == [127, 128, 128, 128]


def test_zerodm_removes_broadband_bursts():
    # A broadband (DM = 0) burst adds the same amount to every channel; after the
    # filter the DM-0 time series is flat up to rounding and the burst is gone.
    nchan, nsamp = 64, 4000
    rfi = synth.RFI(bursts=[(1000, 20, 40.0), (2500, 3, 80.0)])
    X = synth.filterbank(nchan, nsamp, seed=4, rfi=rfi)
    Z = oracle.zerodm(X).astype(np.int64)
    col = Z.sum(axis=0) - 128 * nchan
    assert np.all(np.abs(col) <= nchan // 2)
    raw = X.astype(np.int64).sum(axis=0)
    assert raw[1000:1020].mean() - raw[:900].mean() > 30 * nchan
    # a constant-across-channels input maps to exactly 128 everywhere
    C = np.tile(np.arange(nsamp, dtype=np.int64) % 256, (nchan, 1)).astype(np.uint8)
    assert np.all(oracle.zerodm(C) == 128)


def test_zerodm_keeps_dispersed_pulse():
    # A strongly dispersed pulse puts little power in any one time sample of the
    # DM-0 series, so the filter leaves it (its dedispersed S/N drops by a few %).
    nchan, nsamp, tsamp = 64, 8192, 98.304e-6
    offs = oracle.injection_offsets(nchan, 1000.0, 1500.0, tsamp, 200.0, 1000)
    X = synth.filterbank(nchan, nsamp, seed=6, pulses=[synth.Pulse(offs, 8, synth.pulse_amplitude(20.0, nchan, 8))])
    D = oracle.delay_table(nchan, 1000.0, 1500.0, tsamp, [200.0])
    for arr, lo in [(X, 18.0), (oracle.zerodm(X), 17.0)]:
        Y = oracle.dedisperse(arr, D)
        snr, _ = oracle.boxcar_snr(Y, [8])
        assert snr.max() > lo


@pytest.mark.parametrize("n", [1, 2, 3, 10, 11, 1000, 1001])
def test_robust_is_lower_median(n):
    rng = np.random.default_rng(n)
    Y = rng.integers(0, 50000, size=(3, n), dtype=np.int32)
    med, mad = oracle.row_robust(Y)
    for d in range(3):
        s = np.sort(Y[d].astype(np.int64))
        m = s[(n - 1) // 2]
        assert med[d] == m
        assert mad[d] == np.sort(np.abs(Y[d].astype(np.int64) - m))[(n - 1) // 2]


def test_norm_with_mean_and_std_is_the_plain_snr():
    rng = np.random.default_rng(8)
    Y = rng.normal(5000, 80, size=(4, 3000)).round().astype(np.int32)
    widths = [1, 2, 4, 8, 16]
    S, Q = oracle.rowstats(Y)
    mu = S / Y.shape[1]
    sig = np.array([oracle.row_sigma(S[d], Q[d], Y.shape[1]) for d in range(4)])
    a, ai = oracle.boxcar_snr(Y, widths)
    b, bi = oracle.boxcar_snr_norm(Y, widths, mu, sig)
    fin = np.isfinite(a)
    assert np.array_equal(fin, np.isfinite(b))
    assert np.max(np.abs(a[fin] - b[fin])) < 1e-9
    assert np.array_equal(ai, bi)


def test_tiny_robust_snr_matches_loops():
    rng = np.random.default_rng(12)
    Y = rng.integers(0, 40, size=(2, 9), dtype=np.int32)
    widths = [1, 2, 4]
    snr, bw = oracle.boxcar_snr_robust(Y, widths)
    for d in range(2):
        s = sorted(Y[d].tolist())
        m = s[(9 - 1) // 2]
        mad = sorted(abs(v - m) for v in Y[d].tolist())[(9 - 1) // 2]
        sig = oracle.MAD_TO_SIGMA * mad
        for t in range(9):
            best, bi = -np.inf, -1
            for i, w in enumerate(widths):
                if t + w > 9:
                    continue
                v = (sum(Y[d, t:t + w].tolist()) - w * m) / (sig * np.sqrt(w)) if sig > 0 else 0.0
                if v > best:
                    best, bi = v, i
            assert bw[d, t] == bi
            assert abs(snr[d, t] - best) < 1e-12 or (best == -np.inf and snr[d, t] == -np.inf)


def test_robust_scale_is_sigma_for_gaussian_rows_and_ignores_outliers():
    rng = np.random.default_rng(3)
    Y = rng.normal(10000, 300, size=(8, 200000)).round().astype(np.int32)
    med, mad = oracle.row_robust(Y)
    assert np.all(np.abs(oracle.MAD_TO_SIGMA * mad / 300.0 - 1.0) < 0.02)
    assert np.all(np.abs(med - 10000) < 5)
    # 1 % of strong outliers (RFI) move mean and std a lot, median and MAD little
    Z = Y.copy()
    Z[:, ::100] += 30000
    S, Q = oracle.rowstats(Z)
    std = np.array([oracle.row_sigma(S[d], Q[d], Z.shape[1]) for d in range(8)])
    med2, mad2 = oracle.row_robust(Z)
    assert np.all(std > 4 * 300)
    assert np.all(np.abs(oracle.MAD_TO_SIGMA * mad2 / 300.0 - 1.0) < 0.05)
    assert np.all(np.abs(med2 - 10000) < 20)
