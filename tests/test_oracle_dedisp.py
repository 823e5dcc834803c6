"""Pins for the oracle's brute-force plane, Y[d][t] = sum_c X[c][t+D[d][c]]
(Sec. 2.3): pure-Python brute force, DM 0, impulse response, constant input,
linearity and shift equivariance."""
import numpy as np
import pytest

import oracle
from oracle import brute


def _tiny(rng):
    nchan = int(rng.integers(1, 9))
    nsamp = int(rng.integers(8, 65))
    ndm = int(rng.integers(1, 7))
    X = rng.integers(0, 256, (nchan, nsamp), dtype=np.uint8)
    dmax = int(rng.integers(0, nsamp - 1))
    D = rng.integers(0, dmax + 1, (ndm, nchan)).astype(np.int32)
    return X, D


@pytest.mark.parametrize("seed", range(25))
def test_matches_pure_python_brute_force(seed):
    rng = np.random.default_rng(seed)
    X, D = _tiny(rng)
    nout = X.shape[1] - int(D.max())
    Y = oracle.dedisperse(X, D)
    ref = brute.dedisperse(X.tolist(), D.tolist(), nout)
    assert Y.shape == (D.shape[0], nout)
    assert Y.tolist() == ref


def test_dm_zero_is_channel_sum():
    rng = np.random.default_rng(1)
    X = rng.integers(0, 256, (97, 513), dtype=np.uint8)
    D = oracle.delay_table(97, 1000.0, 1500.0, 1e-3, [0.0, 1.0])
    Y = oracle.dedisperse(X, D)
    nout = 513 - int(D.max())
    assert np.array_equal(Y[0], X[:, :nout].sum(axis=0, dtype=np.int64))


def test_impulse_response_pins_index_and_sign():
    nchan, nsamp = 16, 400
    dms = np.array([0.0, 10.0, 25.0, 40.0])
    D = oracle.delay_table(nchan, 1000.0, 1500.0, 1e-3, dms)
    nout = nsamp - int(D.max())
    for c0, t0 in [(0, 200), (7, 150), (15, 299)]:
        X = np.zeros((nchan, nsamp), dtype=np.uint8)
        X[c0, t0] = 1
        Y = oracle.dedisperse(X, D)
        for d in range(len(dms)):
            expect = np.zeros(nout, dtype=np.int32)
            t = t0 - D[d, c0]
            if 0 <= t < nout:
                expect[t] = 1
            assert np.array_equal(Y[d], expect)


def test_constant_input():
    X = np.full((33, 300), 201, dtype=np.uint8)
    D = oracle.delay_table(33, 1200.0, 1300.0, 5e-4, [0.0, 50.0, 99.0])
    Y = oracle.dedisperse(X, D)
    assert np.all(Y == 33 * 201)


def test_linearity():
    rng = np.random.default_rng(5)
    a = rng.integers(0, 128, (40, 700), dtype=np.uint8)
    b = rng.integers(0, 128, (40, 700), dtype=np.uint8)
    D = oracle.delay_table(40, 1000.0, 1500.0, 2e-4, np.arange(0, 30, 3.0))
    assert np.array_equal(oracle.dedisperse(a + b, D), oracle.dedisperse(a, D) + oracle.dedisperse(b, D))


def test_shift_equivariance():
    rng = np.random.default_rng(9)
    X = rng.integers(0, 256, (24, 900), dtype=np.uint8)
    D = oracle.delay_table(24, 1000.0, 1500.0, 2e-4, np.arange(0, 20, 2.5))
    s = 37
    Y = oracle.dedisperse(X, D)
    Ys = oracle.dedisperse(X[:, s:], D)
    assert np.array_equal(Y[:, s:], Ys)


def test_nout_bounds_checked():
    X = np.zeros((4, 10), dtype=np.uint8)
    D = np.full((1, 4), 10, dtype=np.int32)
    with pytest.raises(ValueError):
        oracle.dedisperse(X, D)


@pytest.mark.parametrize("nchan,hop,nwin", [(16, 120, 4), (7, 37, 3), (33, 1, 5)])
def test_windows_with_hop_nout_tile_the_one_shot_plane(nchan, hop, nwin):
    # Streaming reading of Sec. 2.3 with nout = nsamp - Dmax: windows of Dmax + hop
    # samples that start every hop samples (consecutive windows overlap by Dmax)
    # give planes of hop columns each, and their concatenation is the plane of the
    # whole input, column for column.
    rng = np.random.default_rng(nchan)
    D = oracle.delay_table(nchan, 1000.0, 1500.0, 1e-3, np.arange(0.0, 30.0, 3.0))
    dmax = int(D.max())
    assert dmax > 0
    window = dmax + hop
    total = (nwin - 1) * hop + window
    X = rng.integers(0, 256, (nchan, total), dtype=np.uint8)
    Y = oracle.dedisperse(X, D)
    assert Y.shape[1] == nwin * hop
    parts = [oracle.dedisperse(X[:, k * hop:k * hop + window], D) for k in range(nwin)]
    assert all(p.shape[1] == hop for p in parts)
    assert np.array_equal(np.concatenate(parts, axis=1), Y)
