"""Pins for the oracle's row statistics, boxcar S/N and peak finder (step (iii)
of the standard workflow, Sec. 1; definitions are readings): closed forms,
pure-Python brute force, a statistical pin on white noise."""
import math

import numpy as np
import pytest

import oracle
from oracle import brute


def test_rowstats_against_numpy():
    rng = np.random.default_rng(3)
    Y = rng.integers(0, 1_000_000, (7, 5000)).astype(np.int32)
    S, Q = oracle.rowstats(Y)
    assert np.array_equal(S, Y.astype(np.int64).sum(axis=1))
    assert [int(q) for q in Q] == [int(sum(int(v) * int(v) for v in row)) for row in Y]
    for d in range(7):
        assert abs(oracle.row_sigma(S[d], Q[d], Y.shape[1]) - Y[d].astype(np.float64).std()) < 1e-6 * Y[d].std()


def test_single_spike_closed_form():
    # zero row with one spike h at t0:  sigma = h sqrt(n-1)/n,  snr_1(t0) = sqrt(n-1),
    # any window of width w containing it: (n-w) / (sqrt(n-1) sqrt(w))
    n, t0, h = 1000, 400, 37
    Y = np.zeros((1, n), dtype=np.int32)
    Y[0, t0] = h
    snr, bw = oracle.boxcar_snr(Y, [1])
    assert abs(snr[0, t0] - math.sqrt(n - 1)) < 1e-9
    snr4, _ = oracle.boxcar_snr(Y, [4])
    assert abs(snr4[0, t0 - 3] - (n - 4) / (math.sqrt(n - 1) * 2)) < 1e-9
    # windows without the spike: -mu*w/(sigma sqrt w)
    assert abs(snr[0, 0] - (-1.0 / math.sqrt(n - 1))) < 1e-12


@pytest.mark.parametrize("W", [3, 8, 16])
def test_boxcar_pulse_best_width(W):
    # zero row with a boxcar of width W: best width W, snr = sqrt(n - W) at its start
    n, t0, h = 2000, 700, 5
    Y = np.zeros((1, n), dtype=np.int32)
    Y[0, t0:t0 + W] = h
    widths = [1, 2, 3, 4, 8, 16, 32]
    snr, bw = oracle.boxcar_snr(Y, widths)
    t = int(np.argmax(snr[0]))
    assert t == t0
    assert widths[bw[0, t]] == W
    assert abs(snr[0, t] - math.sqrt(n - W)) < 1e-9


def test_tail_widths_invalid():
    Y = np.arange(50, dtype=np.int32).reshape(1, 50) % 7
    snr, bw = oracle.boxcar_snr(Y, [2, 4])
    assert bw[0, 49] == -1 and snr[0, 49] == -math.inf
    assert bw[0, 48] == 0
    snr, bw = oracle.boxcar_snr(Y, [1, 4])
    assert np.all(bw[0, 47:] == 0)


def test_constant_row_is_zero_snr():
    Y = np.full((2, 64), 9, dtype=np.int32)
    snr, bw = oracle.boxcar_snr(Y, [1, 2, 4])
    assert np.all(snr == 0.0)
    assert np.all(bw[:, :61] == 0)


def test_best_width_exact_tie_goes_to_the_smaller_width():
    # With widths 1 and 4 (sqrt(4) = 2 exactly) a row can tie exactly: at t = 0
    # nout*B_4 - 4*S = 2*(nout*B_1 - S), so snr_4 = (2 num)/(2 den) = snr_1 in IEEE
    # arithmetic.  Row: 16 samples, S = 160 (mean 10), Q = 2400, sigma = sqrt(50);
    # B_1 = 30, B_4 = 80: both S/N are 20 / sqrt(50) = 2 sqrt(2).
    Y = np.array([[30, 20, 20, 10] + [5] * 8 + [10] * 4], dtype=np.int32)
    snr, bw = oracle.boxcar_snr(Y, [1, 4])
    assert snr[0, 0] == pytest.approx(2.0 * math.sqrt(2.0), rel=1e-15)
    assert bw[0, 0] == 0
    bs, bb = brute.boxcar_snr(Y.tolist(), [1, 4])
    assert bb[0][0] == 0 and bs[0][0] == pytest.approx(2.0 * math.sqrt(2.0), rel=1e-15)
    # one count more in the 4-sample window breaks the tie towards width 4
    Y2 = Y.copy()
    Y2[0, 3] += 1
    Y2[0, 15] -= 1
    _, bw2 = oracle.boxcar_snr(Y2, [1, 4])
    assert bw2[0, 0] == 1


@pytest.mark.parametrize("seed", range(8))
def test_snr_matches_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    ndm, n = int(rng.integers(1, 4)), int(rng.integers(5, 60))
    Y = rng.integers(0, 50, (ndm, n)).astype(np.int32)
    widths = sorted(set(int(w) for w in rng.integers(1, 9, 3)))
    snr, bw = oracle.boxcar_snr(Y, widths)
    bs, bb = brute.boxcar_snr(Y.tolist(), widths)
    for d in range(ndm):
        for t in range(n):
            if bs[d][t] == -math.inf:
                assert snr[d, t] == -math.inf
            else:
                assert abs(snr[d, t] - bs[d][t]) <= 1e-9 * max(1.0, abs(bs[d][t]))
                assert bw[d, t] == bb[d][t] or abs(snr[d, t] - bs[d][t]) > 0


def test_white_noise_snr_is_unit_normal():
    rng = np.random.default_rng(11)
    Y = np.rint(rng.normal(5000.0, 40.0, (4, 200_000))).astype(np.int32)
    for w in [1, 4, 16]:
        snr, _ = oracle.boxcar_snr(Y, [w])
        v = snr[:, : Y.shape[1] - w + 1].ravel()
        assert abs(v.mean()) < 0.02
        assert abs(v.std() - 1.0) < 0.02


def test_widths_must_ascend():
    Y = np.zeros((1, 10), dtype=np.int32)
    with pytest.raises(ValueError):
        oracle.boxcar_snr(Y, [2, 1])


@pytest.mark.parametrize("seed", range(10))
def test_peaks_match_brute_force(seed):
    rng = np.random.default_rng(200 + seed)
    ndm, n = int(rng.integers(1, 4)), int(rng.integers(10, 80))
    # coarse values so that ties occur
    snr = rng.integers(0, 6, (ndm, n)).astype(np.float64)
    widths = [1, 2, 4]
    bw = rng.integers(0, 3, (ndm, n)).astype(np.int32)
    bw[0, -1] = -1
    got, total = oracle.peaks(snr, bw, widths, 3.0)
    ref = brute.peaks(snr.tolist(), bw.tolist(), widths, 3.0)
    assert total == len(ref)
    assert got == ref


def test_peaks_tie_goes_to_earliest():
    snr = np.array([[0, 5, 5, 0, 0, 0]], dtype=np.float64)
    bw = np.zeros((1, 6), dtype=np.int32)
    got, _ = oracle.peaks(snr, bw, [1], 4.0)
    assert got == [(0, 1, 1, 5.0)]


def test_peaks_capacity_reports_total():
    snr = np.array([[9, 0, 9, 0, 9, 0, 9]], dtype=np.float64)
    bw = np.zeros((1, 7), dtype=np.int32)
    got, total = oracle.peaks(snr, bw, [1], 8.0, cap=2)
    assert total == 4 and len(got) == 2
