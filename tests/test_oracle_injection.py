"""Pins for the whole oracle search on the 256-channel workload: an injected
dispersed pulse (the paper injects pulses into spectrograms, Sec. 4.1) must be
recovered at its DM and arrival time with the expected width and S/N, and the
clustering / matching rule of Sec. 4.2 must accept it."""
import math

import numpy as np
import pytest

import oracle
from oracle import nms
from paper_2511_02328_gb300 import synth
from conftest import C1, dm_list


@pytest.fixture(scope="module")
def c1_search():
    cfg = C1
    dms = dm_list(cfg)
    W, snr_inj, t0, dm0 = 10, 15.0, 8000, 300.0
    offs = oracle.injection_offsets(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dm0, t0)
    amp = synth.pulse_amplitude(snr_inj, cfg["nchan"], W)
    X = synth.filterbank(cfg["nchan"], cfg["nsamp"], seed=1, pulses=[synth.Pulse(offs, W, amp)])
    D = oracle.delay_table(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms)
    Y = oracle.dedisperse(X, D)
    snr, bw = oracle.boxcar_snr(Y, cfg["widths"])
    return dict(cfg=cfg, dms=dms, X=X, D=D, Y=Y, snr=snr, bw=bw, W=W, t0=t0, snr_inj=snr_inj)


def test_width_rounding():
    # 1 ms at 98.304 us is 10.17 samples -> W = 10
    assert round(1e-3 / C1["tsamp"]) == 10


def test_injected_pulse_recovered(c1_search):
    s = c1_search
    snr, bw, W, t0 = s["snr"], s["bw"], s["W"], s["t0"]
    d, t = np.unravel_index(np.argmax(snr), snr.shape)
    w = s["cfg"]["widths"][bw[d, t]]
    assert d == 300
    assert w == 8
    assert t0 <= t <= t0 + W - w
    # S/N of the best window inside a W-sample boxcar of S/N 15 is 15*sqrt(w/W)
    assert abs(snr[d, t] - s["snr_inj"] * math.sqrt(w / W)) < 2.0
    # off by 10 DM the pulse smears over ~230 samples in the lowest channel
    assert snr[290].max() < snr[d, t] - 3.0
    assert snr[310].max() < snr[d, t] - 3.0


def test_noise_rows_are_normalised(c1_search):
    v = c1_search["snr"][0, :-40]
    # DM 0 row: pure noise, the best of 6 widths is a max over correlated N(0,1)
    assert abs(np.median(v)) < 1.0
    assert v.max() < 6.5


def test_candidates_cluster_and_match(c1_search):
    s = c1_search
    cands, total = oracle.peaks(s["snr"], s["bw"], s["cfg"]["widths"], 8.0)
    assert total == len(cands) > 0
    kept = nms.cluster(cands, s["dms"], s["cfg"]["tsamp"])
    hit, fp = nms.match(kept, [(300.0, s["t0"] * s["cfg"]["tsamp"])], s["dms"], s["cfg"]["tsamp"])
    assert hit == [True]
    assert fp == 0


def test_nms_tolerances():
    dms = np.arange(0, 100, 1.0)
    tsamp = 1e-3
    c = [(50, 1000, 1, 10.0), (60, 1100, 1, 9.0), (71, 1000, 1, 8.0), (50, 1250, 1, 7.0), (30, 1150, 1, 6.0)]
    kept = nms.cluster(c, dms, tsamp)
    # (60,1100): dDM 10, dTOA 0.1 s -> suppressed; (71,1000): dDM 21 -> kept;
    # (50,1250): dTOA 0.25 s -> kept; (30,1150): dDM 20 is not < 20 -> kept
    assert kept == [c[0], c[2], c[3], c[4]]
    kept = nms.cluster(c[:1] + [(45, 1150, 1, 6.0)], dms, tsamp)
    assert kept == c[:1]
