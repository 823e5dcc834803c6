"""Pins for the oracle's square-law time downsampling (Sec. 2.2):
out = min(V*sqrt(S)/sqrt(N*V), V) per bin of N samples with sum S, rounded to
nearest (halves up; reading), exactly in integers."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


def _exact(S, N, V=255):
    """Largest k >= 0 with (k - 1/2)^2 <= V*S/N (round half up of the square
    root), by counting up in exact rationals, then the saturation at V."""
    q = Fraction(V * S, N)
    k = 0
    while (Fraction(2 * (k + 1) - 1, 2)) ** 2 <= q:
        k += 1
    return min(k, V)


def test_single_sample_bins_every_value():
    # D = 1: every 8-bit value maps to round(sqrt(255 * I)).
    X = np.arange(256, dtype=np.uint8).reshape(1, 256)
    out = oracle.downsample_sqlaw(X, 1)
    assert out.shape == (1, 256)
    for i in range(256):
        assert out[0, i] == _exact(i, 1), i
        # no value of 255*I is within reach of a tie: the float formula agrees
        assert out[0, i] == math.floor(math.sqrt(255 * i) + 0.5)
    assert out[0, 0] == 0 and out[0, 255] == 255 and out[0, 1] == 16


def test_constant_bins_and_saturation():
    for c in [0, 1, 17, 128, 200, 254, 255]:
        X = np.full((3, 64), c, dtype=np.uint8)
        out = oracle.downsample_sqlaw(X, 8)
        assert np.all(out == _exact(8 * c, 8))
    # the largest possible mean saturates exactly at V, never beyond
    assert oracle.downsample_sqlaw(np.full((1, 16), 255, np.uint8), 16)[0, 0] == 255


def test_ragged_tail_uses_its_own_count():
    X = np.array([[10, 20, 30, 40, 50, 60, 70, 80, 250, 250]], dtype=np.uint8)
    out = oracle.downsample_sqlaw(X, 4)
    assert out.shape == (1, 3)
    assert out[0].tolist() == [_exact(100, 4), _exact(260, 4), _exact(500, 2)]
    assert out[0, 2] == _exact(250, 1)


@pytest.mark.parametrize("D", [1, 2, 3, 7, 8, 16, 33])
def test_random_bins_exact_rationals(D):
    rng = np.random.default_rng(D)
    X = rng.integers(0, 256, size=(4, 101), dtype=np.uint8)
    out = oracle.downsample_sqlaw(X, D)
    nout = -(-101 // D)
    assert out.shape == (4, nout)
    for c in range(4):
        for k in range(nout):
            w = X[c, k * D:min(101, (k + 1) * D)].astype(int)
            assert out[c, k] == _exact(int(w.sum()), w.size), (c, k)


def test_paper_formula_in_double():
    # The paper's expression V*sqrt(S)/sqrt(N*V) in fp64, rounded half up,
    # agrees wherever it is not within 1e-9 of a half-integer.
    rng = np.random.default_rng(1)
    X = synthetic = rng.normal(128, 12, size=(16, 4096)).round().clip(0, 255).astype(np.uint8)
    for D in (4, 8, 16):
        out = oracle.downsample_sqlaw(synthetic, D).astype(np.int64)
        S = X.reshape(16, -1, D).astype(np.int64).sum(axis=2)
        val = 255.0 * np.sqrt(S) / np.sqrt(D * 255.0)
        frac = val - np.floor(val)
        ok = np.abs(frac - 0.5) > 1e-9
        ref = np.minimum(np.floor(val + 0.5), 255).astype(np.int64)
        assert np.array_equal(out[ok], ref[ok])
        assert ok.mean() > 0.99


def test_monotone_in_the_sum():
    # out is a non-decreasing function of S for a fixed bin size
    vals = [_exact(S, 8) for S in range(0, 8 * 255 + 1, 17)]
    X = np.zeros((len(vals), 8), dtype=np.uint8)
    for i, S in enumerate(range(0, 8 * 255 + 1, 17)):
        q, r = divmod(S, 8)
        X[i, :] = q
        X[i, :r] += 1
    out = oracle.downsample_sqlaw(X, 8)[:, 0]
    assert out.tolist() == vals
    assert np.all(np.diff(out.astype(int)) >= 0)
