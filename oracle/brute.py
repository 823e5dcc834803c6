"""Pure-Python brute force for tiny inputs (test infrastructure only).

Independent restatements of the oracle's definitions, written as nested
Python loops over plain lists, used to pin the C oracle on tiny shapes
(nchan <= 8, nsamp <= 64, ndm <= 6).
"""
import math
from fractions import Fraction

K_DM = Fraction(4148808, 1000)  # s MHz^2 pc^-1 cm^3, Eq. (KDM), unit read as seconds


def exact_delay(dm, fc, fr, tsamp):
    """round(K*DM/tsamp*(1/fc^2 - 1/fr^2)) in exact rational arithmetic, half
    away from zero (Eq. coarse_delay).  Arguments are converted exactly from
    their binary double values, so the only difference from the double oracle
    is the double rounding of the intermediate steps."""
    x = K_DM * Fraction(dm) / Fraction(tsamp) * (1 / Fraction(fc) ** 2 - 1 / Fraction(fr) ** 2)
    n = math.floor(abs(x) + Fraction(1, 2))
    return n if x >= 0 else -n, x


def dedisperse(X, D, nout):
    """Y[d][t] = sum over c of X[c][t + D[d][c]] by direct triple loop."""
    ndm = len(D)
    nchan = len(X)
    Y = [[0] * nout for _ in range(ndm)]
    for d in range(ndm):
        for t in range(nout):
            s = 0
            for c in range(nchan):
                s += int(X[c][t + D[d][c]])
            Y[d][t] = s
    return Y


def boxcar_snr(Y, widths):
    """S/N by the definitions, in Python floats (only for tiny inputs)."""
    out_snr, out_w = [], []
    for row in Y:
        n = len(row)
        mu = Fraction(sum(row), n)
        var = sum((Fraction(v) - mu) ** 2 for v in row) / n
        sigma = math.sqrt(var)
        srow, wrow = [], []
        for t in range(n):
            best, bi = -math.inf, -1
            for i, w in enumerate(widths):
                if t + w > n:
                    continue
                B = sum(row[t:t + w])
                snr = float((B - w * mu) / Fraction(sigma) / Fraction(math.sqrt(w))) if sigma > 0 else 0.0
                if snr > best:
                    best, bi = snr, i
            srow.append(best)
            wrow.append(bi)
        out_snr.append(srow)
        out_w.append(wrow)
    return out_snr, out_w


def peaks(snr, bw, widths, thresh):
    """Local maxima along t within +-w (ties to the earliest t), above thresh."""
    res = []
    for d, row in enumerate(snr):
        n = len(row)
        for t in range(n):
            if not row[t] >= thresh or bw[d][t] < 0:
                continue
            w = widths[bw[d][t]]
            left = [row[u] for u in range(max(0, t - w), t)]
            right = [row[u] for u in range(t + 1, min(n, t + w + 1))]
            if all(row[t] > v for v in left) and all(row[t] >= v for v in right):
                res.append((d, t, w, row[t]))
    return res


def exact_shift(ddm, inv_f2, fr, tsamp):
    """round(K*dDM/tsamp*(inv_f2 - 1/fr^2)) in exact rational arithmetic, half
    away from zero: Eq. (residual) with 1/F_s^2 given directly (a Fraction)."""
    x = K_DM * Fraction(ddm) / Fraction(tsamp) * (inv_f2 - 1 / Fraction(fr) ** 2)
    n = math.floor(abs(x) + Fraction(1, 2))
    return n if x >= 0 else -n, x


def subband_dedisperse(X, Dc, first, R, n0, nout):
    """Eqs. (stage1) and (stage2) by direct loops: for fine DM m in coarse
    group j = m // n0, Y[m][v] = sum over subbands s of I(j, s, v + R[m][s]),
    I(j, s, u) = sum over channels c of s of X[c][u + Dc[j][c]], with X taken
    as zero outside the data."""
    nsamp = len(X[0])
    nsub = len(first) - 1
    Y = []
    for m in range(len(R)):
        j = m // n0
        row = []
        for v in range(nout):
            total = 0
            for s in range(nsub):
                u = v + R[m][s]
                for c in range(first[s], first[s + 1]):
                    t = u + Dc[j][c]
                    if 0 <= t < nsamp:
                        total += int(X[c][t])
            row.append(total)
        Y.append(row)
    return Y
