"""Pins for the oracle's DM-time slice gridding (Sec. 2.4): slicing, exact
pixel-area averaging, Lanczos-4 resampling and the 8-bit normalisation."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import grid


def test_slicing_of_the_benchmark_plane():
    # T_slice = 0.5 s (the paper's T_grid) on the 4096-channel plane (nout 215,261).
    n_s, S, rng = grid.slices(215261, 0.5, 49.152e-6)
    assert n_s == math.ceil(0.5 / 49.152e-6) == 10173
    assert S == 22 and rng[0] == (0, 10173) and rng[-1] == (21 * 10173, 215261)
    assert sum(c1 - c0 for c0, c1 in rng) == 215261


@pytest.mark.parametrize("n,M", [(1001, 512), (10173, 512), (7, 3), (512, 512), (3, 5)])
def test_overlap_matrix_partitions(n, M):
    R = grid.overlap_matrix(n, M)
    assert np.all(R.sum(axis=1) == n)       # every output pixel covers n scaled units
    assert np.all(R.sum(axis=0) == M)       # every input pixel is spread over M units


def test_area_is_block_mean_for_integer_factors():
    rng = np.random.default_rng(1)
    X = rng.integers(0, 10 ** 6, size=(64, 96))
    W = grid.area_weights(X, 16)
    U = W / (64 * 96)
    assert np.allclose(U, X.reshape(16, 4, 16, 6).mean(axis=(1, 3)), rtol=0, atol=1e-9)
    assert W.sum() == 16 * 16 * X.sum()


def test_area_exact_rationals_tiny():
    # explicit interval overlaps in exact rationals, independent of the matrix form
    rng = np.random.default_rng(2)
    X = rng.integers(0, 1000, size=(5, 7))
    M = 3
    W = grid.area_weights(X, M)
    for i in range(M):
        for j in range(M):
            acc = Fraction(0)
            for r in range(5):
                ry = max(0, min(Fraction(i + 1, M) * 5, r + 1) - max(Fraction(i, M) * 5, r))
                for c in range(7):
                    cx = max(0, min(Fraction(j + 1, M) * 7, c + 1) - max(Fraction(j, M) * 7, c))
                    acc += ry * cx * int(X[r, c])
            # U = pixel-area mean = acc / (output pixel area (5/M)(7/M))
            assert Fraction(int(W[i, j]), 5 * 7) == acc / (Fraction(5, M) * Fraction(7, M))


def test_lanczos_identity_constant_and_kernel():
    A = grid.lanczos4_matrix(9, 9)
    assert np.allclose(A, np.eye(9), atol=1e-12)          # integer offsets: L(0) = 1, L(k) = 0
    B = grid.lanczos4_matrix(5, 13)
    assert np.allclose(B.sum(axis=1), 1.0)                 # normalised: constants are preserved
    t = 0.5
    assert np.sinc(t) * np.sinc(t / 4) == pytest.approx((2 / math.pi) * math.sin(math.pi / 8) / (math.pi / 8))
    # mirror symmetry of the up-sampling weights
    assert np.allclose(B, B[::-1, ::-1], atol=1e-12)
    # an interior row follows the closed form L(t) = 4 sin(pi t) sin(pi t / 4) / (pi t)^2
    C = grid.lanczos4_matrix(10, 20)
    x = (10 + 0.5) * 10 / 20 - 0.5                         # 4.75: taps 1 .. 8, no clamping
    L = np.array([4 * math.sin(math.pi * (x - k)) * math.sin(math.pi * (x - k) / 4) / (math.pi * (x - k)) ** 2
                  for k in range(1, 9)])
    assert np.allclose(C[10, 1:9], L / L.sum(), atol=1e-12)
    assert np.all(C[10, [0, 9]] == 0)


def test_gray_levels():
    W = np.array([[3, 10], [17, 3]], dtype=np.int64)
    Y = grid.gray_exact(W)
    assert Y.tolist() == [[0, 128], [255, 0]]             # 255 * 7/14 = 127.5 rounds up
    assert np.all(grid.gray_exact(np.full((4, 4), 9)) == 0)
    rng = np.random.default_rng(3)
    W = rng.integers(-10 ** 12, 10 ** 12, size=(64, 64))
    lo, hi = W.min(), W.max()
    f = 255.0 * (W - lo) / (hi - lo)
    ok = np.abs(f - np.floor(f) - 0.5) > 1e-6
    assert np.array_equal(grid.gray_exact(W)[ok], grid.to_gray(W.astype(np.float64), (lo, hi), eps=0)[ok])
    # the Lanczos path keeps eps: a slice that is constant up to rounding maps to 0
    U = np.full((8, 8), 42.0) + np.random.default_rng(5).normal(0, 1e-12, (8, 8))
    assert np.all(grid.to_gray(U, (U.min(), U.max())) == 0)


def test_path_selection():
    rng = np.random.default_rng(4)
    assert grid.grid_slice(rng.integers(0, 100, size=(600, 700)), M=512)[1] == "area"
    assert grid.grid_slice(rng.integers(0, 100, size=(600, 300)), M=512)[1] == "lanczos4"
    assert grid.grid_slice(rng.integers(0, 100, size=(512, 700)), M=512)[1] == "lanczos4"   # N_DM = M: no shrink
    assert grid.grid_slice(rng.integers(0, 100, size=(20, 30)), M=16)[1] == "area"
    Y, path = grid.grid_slice(rng.integers(0, 100, size=(10, 30)), M=16)
    assert path == "lanczos4" and Y.min() == 0 and Y.max() == 255
