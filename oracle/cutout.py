"""Cut-out oracle (test infrastructure only).

The paper slices the DM-time plane into images for its detector (Sec. 2.4:
resampling to M x M and the per-slice min-max normalisation of its gridding
equation).  The build's classifier instead looks at two 64 x 64 cut-outs
around each candidate (reading; the paper's YOLO images need its weights):

  time bins    b = max(1, w // 2) samples, 64 bins, bin j covers output samples
               [t - 32 b + j b, t - 32 b + (j + 1) b); samples outside [0, nout)
               contribute 0
  DM-time      row i = plane row d - 32 + i (rows outside [0, ndm) are zero),
               value = sum of the row over the bin
  freq-time    group g = channels [g * nchan/64, (g + 1) * nchan/64), value =
               sum over the group's channels c and the bin's samples s of
               X[c][s + D[d][c]] (the data dedispersed at the candidate's DM)
  normalise    each cut-out separately: with lo / hi its min / max (exact
               integers), v' = float32(v - lo) / (float32(hi - lo) + 1e-6f),
               IEEE float32 division, then rounded to bfloat16 (nearest even).

Output [2][64][64] float32 holding bfloat16 values: channel 0 DM-time, 1 freq-time.
"""
import numpy as np

SIDE = 64


def bf16_round(x):
    """float32 -> bfloat16 (round to nearest, ties to even) -> float32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _normalise(v):
    v = np.asarray(v, dtype=np.int64)
    lo, hi = int(v.min()), int(v.max())
    num = (v - lo).astype(np.float32)
    den = np.float32(hi - lo) + np.float32(1e-6)
    return bf16_round(num / den)


def bins(t, w, nout):
    b = max(1, int(w) // 2)
    starts = int(t) - 32 * b + b * np.arange(SIDE)
    return b, starts


def dm_time(plane, d, t, w):
    ndm, nout = plane.shape
    b, starts = bins(t, w, nout)
    out = np.zeros((SIDE, SIDE), dtype=np.int64)
    for i in range(SIDE):
        r = d - 32 + i
        if r < 0 or r >= ndm:
            continue
        for j in range(SIDE):
            lo, hi = max(0, starts[j]), min(nout, starts[j] + b)
            if lo < hi:
                out[i, j] = int(plane[r, lo:hi].astype(np.int64).sum())
    return out


def freq_time(X, D, d, t, w, nout):
    nchan = X.shape[0]
    if nchan % SIDE:
        raise ValueError("nchan must be a multiple of 64")
    gsz = nchan // SIDE
    b, starts = bins(t, w, nout)
    out = np.zeros((SIDE, SIDE), dtype=np.int64)
    for g in range(SIDE):
        for c in range(g * gsz, (g + 1) * gsz):
            row = X[c].astype(np.int64)
            dc = int(D[d, c])
            for j in range(SIDE):
                lo, hi = max(0, starts[j]), min(nout, starts[j] + b)
                if lo < hi:
                    out[g, j] += int(row[lo + dc:hi + dc].sum())
    return out


def cutouts(X, D, plane, cands):
    """cands: iterable of (dm_idx, t, width).  Returns float32 [n][2][64][64]."""
    nout = plane.shape[1]
    res = []
    for (d, t, w) in cands:
        a = _normalise(dm_time(plane, int(d), int(t), int(w)))
        f = _normalise(freq_time(X, D, int(d), int(t), int(w), nout))
        res.append(np.stack([a, f]))
    return np.array(res, dtype=np.float32).reshape(-1, 2, SIDE, SIDE)
