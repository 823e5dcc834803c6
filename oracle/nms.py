"""Candidate clustering and the true-positive matching rule (test
infrastructure only).

Sec. 4.2 of the paper counts a detection as a true positive when
|DM_det - DM_true| < 20 pc cm^-3 and |TOA_det - TOA_true| < 0.2 s, with TOA
referenced to the top of the band.  The same tolerance is used here to merge
candidates into clusters (greedy, strongest first) and to match clusters to
injected pulses.
"""

DM_TOL = 20.0
TOA_TOL = 0.2


def cluster(cands, dm_list, tsamp, dm_tol=DM_TOL, toa_tol=TOA_TOL):
    """Greedy suppression: visit candidates by (snr desc, dm_idx asc, t asc);
    keep one unless a kept candidate lies within both tolerances.
    cands: iterable of (dm_idx, t, width, snr); t is the sample index of the
    arrival at f_ref.  Returns the kept candidates in visiting order."""
    order = sorted(cands, key=lambda c: (-c[3], c[0], c[1]))
    kept = []
    for c in order:
        dm, toa = dm_list[c[0]], c[1] * tsamp
        ok = True
        for k in kept:
            if abs(dm_list[k[0]] - dm) < dm_tol and abs(k[1] * tsamp - toa) < toa_tol:
                ok = False
                break
        if ok:
            kept.append(c)
    return kept


def match(clusters, injections, dm_list, tsamp, dm_tol=DM_TOL, toa_tol=TOA_TOL):
    """injections: list of (dm, toa_seconds).  Returns (recalled flags, number
    of clusters that match no injection)."""
    hit = [False] * len(injections)
    fp = 0
    for c in clusters:
        dm, toa = dm_list[c[0]], c[1] * tsamp
        m = False
        for i, (idm, itoa) in enumerate(injections):
            if abs(idm - dm) < dm_tol and abs(itoa - toa) < toa_tol:
                hit[i] = True
                m = True
        if not m:
            fp += 1
    return hit, fp
