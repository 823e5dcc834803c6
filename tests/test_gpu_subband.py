"""Parity of the two-stage subband dedispersion (Sec. 2.3, Eqs. stage1,
residual, stage2) with the CPU oracle, through the C ABI.

Tables (partition, F_s, coarse delays, residual shifts, effective delays):
identical.  Plane and row sums: bit-exact, for the two-stage kernels and for
the brute-force kernels on the effective delays."""
import os

import numpy as np
import pytest

import oracle
from conftest import C1, dm_list
from paper_2511_02328_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


C2_LIKE = dict(nchan=4096, f_lo=1000.0, f_hi=1500.0, tsamp=49.152e-6, nsamp=1 << 18)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _plan(nchan, f_lo, f_hi, tsamp, dms, n0, nsub, mode, block_len=0, kernel=None):
    from paper_2511_02328_gb300.search import Plan
    old = os.environ.get("AFGB_DEDISP_KERNEL")
    try:
        if kernel is not None:
            os.environ["AFGB_DEDISP_KERNEL"] = kernel
        return Plan(nchan, f_lo, f_hi, tsamp, dms, subband=dict(n0=n0, nsub=nsub, fs_mode=mode, block_len=block_len))
    finally:
        if old is None:
            os.environ.pop("AFGB_DEDISP_KERNEL", None)
        else:
            os.environ["AFGB_DEDISP_KERNEL"] = old


def _run(p, X):
    x = torch.from_numpy(X).cuda()
    stats = torch.empty((p.ndm, 2), dtype=torch.int64, device="cuda")
    Y = p.dedisperse(x, stats=stats)
    torch.cuda.synchronize()
    from paper_2511_02328_gb300 import _lib
    _lib.af_plan_check(p.handle)
    return Y.cpu().numpy(), stats.cpu().numpy()


# nchan, nsamp, f_lo, f_hi, tsamp, dms, n0, nsub, mode, block_len
CASES = [
    (64, 6000, 1000.0, 1500.0, 98.304e-6, np.arange(0.0, 60.0, 1.0), 4, 8, 1, 0),
    (48, 5000, 1500.0, 1000.0, 98.304e-6, np.arange(0.0, 40.0, 0.7), 5, 5, 0, 0),
    (33, 7001, 1200.0, 1450.0, 65.536e-6, np.array([0.0, 0.0, 1.0, 5.0, 5.5, 9.0, 30.0]), 3, 4, 1, 0),
    (255, 20011, 1000.0, 1500.0, 98.304e-6, np.arange(0.0, 150.0, 1.0), 8, 17, 1, 8192),
    (256, 1 << 15, 1000.0, 1500.0, 98.304e-6, np.arange(0.0, 501.0, 1.0), 8, 16, 1, 0),
    (256, 1 << 15, 1000.0, 1500.0, 98.304e-6, np.arange(0.0, 501.0, 1.0), 16, 32, 0, 4096),
    (300, 30000, 1000.0, 1500.0, 98.304e-6, np.arange(0.0, 200.0, 2.0), 32, 1, 1, 0),
    (520, 20000, 1000.0, 1500.0, 98.304e-6, np.arange(0.0, 100.0, 1.0), 7, 2, 1, 0),
    (4096, 20000, 1000.0, 1500.0, 49.152e-6, np.arange(0.0, 40.0, 1.0), 8, 64, 1, 0),
    (100, 9000, 1000.0, 1500.0, 98.304e-6, np.arange(0.0, 70.0, 0.5), 1, 10, 0, 0),
    # residual-shift tables too large for shared memory (stage 2 reads them from global memory)
    (1200, 9000, 1000.0, 1500.0, 98.304e-6, np.arange(0.0, 40.0, 1.0), 8, 600, 1, 0),
    (1024, 9000, 1500.0, 1000.0, 98.304e-6, np.arange(0.0, 30.0, 1.0), 6, 1024, 0, 0),
]
IDS = ["%dch-n0%d-sub%d" % (c[0], c[6], c[7]) for c in CASES]


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_tables_identical(case):
    nchan, nsamp, f_lo, f_hi, tsamp, dms, n0, nsub, mode, L = case
    p = _plan(nchan, f_lo, f_hi, tsamp, dms, n0, nsub, mode, L)
    tab = oracle.subband_tables(nchan, f_lo, f_hi, tsamp, dms, n0, nsub, mode)
    info = p.subband_info()
    assert info["n0"] == n0 and info["nsub"] == nsub and info["ncoarse"] == tab["Dc"].shape[0]
    assert np.array_equal(info["first"], tab["first"])
    assert np.array_equal(info["F"], tab["F"])          # the same IEEE double sequence
    assert np.array_equal(info["Dc"], tab["Dc"])
    assert np.array_equal(info["R"], tab["R"])
    Deff = oracle.subband_effective_delays(tab)
    assert np.array_equal(p.delays(), Deff)
    assert p.dmax == int(Deff.max())
    if L:
        assert info["block_len"] == L
    else:
        assert info["block_len"] % 4096 == 0 and 4096 <= info["block_len"] <= (1 << 18)
    p.close()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_plane_bit_exact(case):
    nchan, nsamp, f_lo, f_hi, tsamp, dms, n0, nsub, mode, L = case
    rng = np.random.default_rng(nchan + n0)
    X = rng.integers(0, 256, size=(nchan, nsamp), dtype=np.uint8)
    tab = oracle.subband_tables(nchan, f_lo, f_hi, tsamp, dms, n0, nsub, mode)
    Yref = oracle.subband_dedisperse(X, tab)
    S, Q = oracle.rowstats(Yref)
    p = _plan(nchan, f_lo, f_hi, tsamp, dms, n0, nsub, mode, L)
    Y, st = _run(p, X)
    assert Y.shape == Yref.shape
    assert np.array_equal(Y, Yref)
    assert np.array_equal(st[:, 0], S) and np.array_equal(st[:, 1], Q)
    p.close()


@pytest.mark.parametrize("kernel", ["brute", "simple"])
def test_brute_kernels_on_effective_delays(kernel):
    # The brute-force kernels fed the plan's effective delays give the same plane.
    nchan, nsamp, f_lo, f_hi, tsamp, dms, n0, nsub, mode, L = CASES[4]
    rng = np.random.default_rng(3)
    X = rng.integers(0, 256, size=(nchan, nsamp), dtype=np.uint8)
    tab = oracle.subband_tables(nchan, f_lo, f_hi, tsamp, dms, n0, nsub, mode)
    Yref = oracle.subband_dedisperse(X, tab)
    p = _plan(nchan, f_lo, f_hi, tsamp, dms, n0, nsub, mode, L, kernel=kernel)
    Y, _ = _run(p, X)
    assert np.array_equal(Y, Yref)
    p.close()


def test_n0_one_equals_brute_force_plan():
    from paper_2511_02328_gb300.search import Plan
    cfg = C1
    dms = dm_list(cfg)
    X = synth.filterbank(cfg["nchan"], cfg["nsamp"], seed=9)
    p = _plan(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms, 1, 16, 1)
    q = Plan(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms)
    Y1, _ = _run(p, X)
    Y2, _ = _run(q, X)
    assert np.array_equal(Y1, Y2)
    p.close()
    q.close()


def test_repeated_calls_and_two_plans():
    # Scratch lives in each plan: two plans alternating on one stream agree with
    # themselves and with the oracle.
    nchan, nsamp, f_lo, f_hi, tsamp, dms, n0, nsub, mode, L = CASES[0]
    rng = np.random.default_rng(4)
    X1 = rng.integers(0, 256, size=(nchan, nsamp), dtype=np.uint8)
    X2 = rng.integers(0, 256, size=(nchan, nsamp), dtype=np.uint8)
    tab = oracle.subband_tables(nchan, f_lo, f_hi, tsamp, dms, n0, nsub, mode)
    p1 = _plan(nchan, f_lo, f_hi, tsamp, dms, n0, nsub, mode)
    p2 = _plan(nchan, f_lo, f_hi, tsamp, dms, n0, nsub, mode, 4096)
    for _ in range(2):
        assert np.array_equal(_run(p1, X1)[0], oracle.subband_dedisperse(X1, tab))
        assert np.array_equal(_run(p2, X2)[0], oracle.subband_dedisperse(X2, tab))
    p1.close()
    p2.close()


def test_search_finds_pulse_between_coarse_dms():
    # Whole search on a subband plan: the injected pulse (DM 301, between the
    # coarse DMs 296 and 304) is a candidate near its DM and arrival time.
    from paper_2511_02328_gb300 import _lib
    cfg = C1
    dms = dm_list(cfg)
    offs = oracle.injection_offsets(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], 301.0, 9000)
    X = synth.filterbank(cfg["nchan"], cfg["nsamp"], seed=3,
                         pulses=[synth.Pulse(offs, 10, synth.pulse_amplitude(15.0, cfg["nchan"], 10))])
    p = _plan(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms, 8, 32, 1)
    _lib.af_search_reserve(p.handle, cfg["nsamp"], 4096)
    cands, n = _lib.af_search(p.handle, X, cfg["nsamp"], cfg["widths"], 8.0, 4096)
    assert n >= 1
    best = cands[np.argmax(cands["snr"])]
    assert abs(dms[best["dm_idx"]] - 301.0) <= 3
    assert abs(int(best["abs_sample"]) - 9000) <= 10
    # and the oracle's S/N on its own subband plane agrees
    tab = oracle.subband_tables(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms, 8, 32, 1)
    Yref = oracle.subband_dedisperse(X, tab)
    snr, _ = oracle.boxcar_snr(Yref[best["dm_idx"]:best["dm_idx"] + 1], cfg["widths"])
    assert abs(float(best["snr"]) - snr.max()) <= 1e-5 * max(1.0, snr.max())
    p.close()


def test_argument_errors():
    from paper_2511_02328_gb300 import _lib
    bad = [
        dict(dm_list=[0.0, 2.0, 1.0], n0=2, nsub=4, mode=1),      # decreasing DMs
        dict(dm_list=[0.0, 1.0], n0=0, nsub=4, mode=1),
        dict(dm_list=[0.0, 1.0], n0=33, nsub=4, mode=1),
        dict(dm_list=[0.0, 1.0], n0=2, nsub=65, mode=1),          # more subbands than channels
        dict(dm_list=[0.0, 1.0], n0=2, nsub=4, mode=2),
    ]
    for b in bad:
        with pytest.raises(_lib.AFError) as ei:
            _lib.af_plan_subband(64, 1000.0, 1500.0, 1e-4, b["dm_list"], b["n0"], b["nsub"], b["mode"])
        assert ei.value.code == _lib.AF_EINVAL
    p = _lib.af_plan(64, 1000.0, 1500.0, 1e-4, [0.0, 1.0])
    with pytest.raises(_lib.AFError):
        _lib.af_plan_subband_info(p)
    _lib.af_plan_destroy(p)


def test_full_size_sampled_rows():
    # 4096 channels x 2^18 samples, DMs 0..1000, n0 = 8, 64 subbands, the block
    # length the bench uses: sampled rows against the brute-force oracle on the
    # effective delays, plus exact row sums of those rows.
    nchan, nsamp = 4096, 1 << 18
    dms = np.arange(0.0, 1001.0, 1.0)
    X = synth.filterbank(nchan, nsamp, seed=2)
    p = _plan(nchan, 1000.0, 1500.0, 49.152e-6, dms, 8, 64, 1, 1 << 18)
    Y, st = _run(p, X)
    tab = oracle.subband_tables(nchan, 1000.0, 1500.0, 49.152e-6, dms, 8, 64, 1)
    Deff = oracle.subband_effective_delays(tab)
    rows = [0, 1, 7, 8, 500, 503, 999, 1000]
    Yref = oracle.dedisperse(X, Deff[rows], Y.shape[1])
    assert np.array_equal(Y[rows], Yref)
    S, Q = oracle.rowstats(Yref)
    assert np.array_equal(st[rows, 0], S) and np.array_equal(st[rows, 1], Q)
    p.close()


@pytest.mark.slow
def test_snr_loss_of_twenty_pulses_within_the_smearing_bound():
    """The benchmark's subband setting (n0 = 8, 64 subbands of 64 channels,
    1/f^2 centres) on the 4096-channel workload with its 20 injected pulses
    (DM U(50, 1000), width log-U(0.2, 10) ms, S/N U(6, 30), placed by the
    oracle's injector): every pulse the brute-force plane finds keeps the
    fraction of its brute-force S/N that the smearing of Eq. (sb_smear) allows.
    A pulse of W samples whose subband delays spread it over d more samples
    (d = the largest 2 K |dDM| df_s / F_s^3 of its subbands, in samples, plus
    two samples of rounding) keeps at least sqrt(W / (W + d)) of its matched-
    filter S/N; the S/N measurements carry unit noise, allowed for as 3 /
    S/N_brute.  Best S/N per pulse = the largest boxcar S/N within |dDM| < 20
    and |dTOA| < 0.2 s (Sec. 4.2)."""
    from paper_2511_02328_gb300 import _lib, synth
    from paper_2511_02328_gb300.search import Plan
    cfg = dict(C2_LIKE)
    nchan, f_lo, f_hi, tsamp, nsamp = cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], cfg["nsamp"]
    dms = np.arange(0.0, 1001.0, 1.0)
    widths = [1, 2, 4, 8, 16, 32, 64, 128, 256]
    pp = synth.pulse_params(20, 13012, (50.0, 1000.0), (0.2e-3, 10e-3), (6.0, 30.0),
                            (0.5, (nsamp - 50000) * tsamp - 0.5), 0.45, tsamp)
    pulses = [synth.Pulse(oracle.injection_offsets(nchan, f_lo, f_hi, tsamp, p["dm"], p["t0"]), p["width"],
                          synth.pulse_amplitude(p["snr"], nchan, p["width"])) for p in pp]
    x = torch.from_numpy(synth.filterbank(nchan, nsamp, seed=12012, pulses=pulses)).cuda()
    n0, nsub = 8, 64
    tab = oracle.subband_tables(nchan, f_lo, f_hi, tsamp, dms, n0, nsub, oracle.FS_INVSQ)
    best = {}
    for name, plan in (("brute", Plan(nchan, f_lo, f_hi, tsamp, dms)),
                       ("subband", Plan(nchan, f_lo, f_hi, tsamp, dms,
                                        subband=dict(n0=n0, nsub=nsub, fs_mode=_lib.AF_FS_INVSQ, block_len=nsamp)))):
        plane = plan.dedisperse(x)
        snr, _ = plan.boxcar_snr(plane, widths)
        torch.cuda.synchronize()
        if name == "subband":
            _lib.af_plan_check(plan.handle)
        vals = []
        for p in pp:
            rows = np.nonzero(np.abs(dms - p["dm"]) < 20.0)[0]
            half = int(0.2 / tsamp)
            t0, t1 = max(0, p["t0"] - half), min(plane.shape[1], p["t0"] + half + 1)
            vals.append(float(snr[rows[0]:rows[-1] + 1, t0:t1].max().item()))
        best[name] = np.array(vals)
        del plane, snr
        plan.close()
    # the smearing of Eq. (sb_smear) at each pulse's nearest fine DM, in samples
    f = f_lo + (np.arange(nchan) + 0.5) * (f_hi - f_lo) / nchan
    width = (f_hi - f_lo) / nchan * np.diff(tab["first"])
    ratios, checked = [], 0
    for i, p in enumerate(pp):
        m = int(np.argmin(np.abs(dms - p["dm"])))
        ddm = abs(dms[m] - dms[(m // n0) * n0])
        d = float(np.max(2.0 * 4.148808e3 * ddm * width / tab["F"] ** 3)) / tsamp + 2.0
        sb, ss = best["brute"][i], best["subband"][i]
        if sb < 8.0:                      # not a detection of the brute-force plane
            continue
        checked += 1
        ratios.append(ss / sb)
        bound = np.sqrt(p["width"] / (p["width"] + d)) - 3.0 / sb
        assert ss / sb >= bound, (i, p, ss, sb, d, bound)
    print("subband / brute-force S/N on %d pulses: mean %.4f min %.4f" % (checked, np.mean(ratios), np.min(ratios)))
    assert checked >= 10                  # of 20 injected at S/N U(6, 30)
    assert np.mean(ratios) >= 0.95
