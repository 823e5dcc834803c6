"""DM-time slice gridding for an image detector (Sec. 2.4, "Griding and
Rendering") -- test infrastructure only (see oracle/__init__.py).

Plain numpy restatement of the paper's steps, in its notation:
  n_s = ceil(T_slice / t_samp),  S = ceil(N_t / n_s)        (slice length and count)
  slice s = plane columns [s n_s, min((s+1) n_s, N_t))
  U^(s) = the slice resampled to M x M (M = 512): area averaging when both
          dimensions shrink (N_DM > M and n_s^(s) > M), Lanczos-4 otherwise
  Y^(s) = round(255 (U - u_min) / (u_max - u_min + eps))   (8-bit grayscale)
The pseudo-colour map applied after Y (a fixed 256-entry table) is not part of
this restatement.

Readings (the paper names OpenCV's interpolations and gives no formulas):
  * area averaging is the exact pixel-area mean: output pixel (i, j) covers
    input rows [i h / M, (i+1) h / M) and columns [j w / M, (j+1) w / M); in
    units scaled by M every overlap length is an integer, so
    W = Rw X Cw^T (Rw[i][r] = |[i h, (i+1) h) & [r M, (r+1) M)|, likewise Cw)
    is exact and U = W / (h w);
  * Lanczos-4: separable, source coordinate x = (i + 0.5) h / M - 0.5, taps
    floor(x) - 3 .. floor(x) + 4 with weights L(x - k), L(t) = sinc(t) sinc(t/4),
    normalised to sum 1, indices clamped to the image (replicated border);
  * Y = floor(255 (U - u_min) / (u_max - u_min + eps) + 1/2) (round half up)
    with eps = 1e-6 on the Lanczos path, where U is a floating-point sum and a
    constant slice would otherwise normalise its rounding noise; on the area
    path U = W / (h w) is exact and the ratio is taken from the integers W
    without eps (Y = 0 for a constant slice).
"""
import math

import numpy as np

M_DEFAULT = 512


def slices(n_t, t_slice, tsamp):
    """(n_s, S, [(c0, c1), ...]) of the slicing of n_t plane columns."""
    n_s = int(math.ceil(t_slice / tsamp))
    S = int(math.ceil(n_t / n_s))
    return n_s, S, [(s * n_s, min((s + 1) * n_s, n_t)) for s in range(S)]


def overlap_matrix(n, M):
    """int64 [M][n]: length of [i n, (i+1) n) & [r M, (r+1) M) (units scaled by M)."""
    i = np.arange(M, dtype=np.int64)[:, None]
    r = np.arange(n, dtype=np.int64)[None, :]
    lo = np.maximum(i * n, r * M)
    hi = np.minimum((i + 1) * n, (r + 1) * M)
    return np.maximum(hi - lo, 0)


def area_weights(X, M):
    """Exact W = Rw X Cw^T (int64) of the pixel-area mean; U = W / (h w).
    The overlap matrices are sparse (a few entries per row), so the two
    integer products are taken with scipy's sparse matrix product."""
    from scipy import sparse
    X = np.asarray(X, dtype=np.int64)
    h, w = X.shape
    Rw = sparse.csr_matrix(overlap_matrix(h, M))
    CwT = sparse.csr_matrix(overlap_matrix(w, M).T)
    XC = (sparse.csr_matrix(X) @ CwT).toarray().astype(np.int64)
    return (Rw @ XC).astype(np.int64)


def lanczos4_matrix(n, M):
    """float64 [M][n]: normalised Lanczos-4 weights with a replicated border."""
    A = np.zeros((M, n))
    for i in range(M):
        x = (i + 0.5) * n / M - 0.5
        k0 = math.floor(x)
        taps = [(k, np.sinc(x - k) * np.sinc((x - k) / 4.0)) for k in range(k0 - 3, k0 + 5)]
        tot = sum(v for _, v in taps)
        for k, v in taps:
            A[i, min(max(k, 0), n - 1)] += v / tot
    return A


EPS = 1e-6


def to_gray(num, den_lo_hi, eps=EPS):
    """Y = floor(255 (v - lo) / (hi - lo + eps) + 1/2) (0 where hi == lo and eps == 0)."""
    v, lo, hi = num, den_lo_hi[0], den_lo_hi[1]
    if hi == lo and eps == 0:
        return np.zeros(v.shape, dtype=np.uint8)
    return np.floor(255.0 * (v - lo) / (hi - lo + eps) + 0.5).astype(np.uint8)


def gray_exact(W):
    """The area path's Y from the exact integers W: floor((510 (W - lo) + (hi - lo)) / (2 (hi - lo)))."""
    lo, hi = int(W.min()), int(W.max())
    if hi == lo:
        return np.zeros(W.shape, dtype=np.uint8)
    num = [(510 * (int(v) - lo) + (hi - lo)) // (2 * (hi - lo)) for v in W.ravel()]
    return np.array(num, dtype=np.int64).reshape(W.shape).astype(np.uint8)


def grid_slice(X, M=M_DEFAULT):
    """(Y uint8 [M][M], path) of one plane slice X [N_DM][n]."""
    h, w = X.shape
    if h > M and w > M:
        return gray_exact(area_weights(X, M)), "area"
    U = lanczos4_matrix(h, M) @ np.asarray(X, dtype=np.float64) @ lanczos4_matrix(w, M).T
    return to_gray(U, (U.min(), U.max())), "lanczos4"


def grid(plane, t_slice, tsamp, M=M_DEFAULT):
    """uint8 [S][M][M]: every slice of the DM-time plane, gridded."""
    n_s, S, rng = slices(plane.shape[1], t_slice, tsamp)
    return np.stack([grid_slice(plane[:, c0:c1], M)[0] for c0, c1 in rng])
