"""The seeded input generator against its recipe: noise N(128, 12) rounded half
to even and clipped to [0, 255]; a boxcar pulse of integrated S/N `snr` over
nchan channels and W samples adds snr * sigma / sqrt(nchan * W) per sample;
the RFI shapes of Sec. 4.4; pulse parameters drawn within their ranges."""
import numpy as np
import pytest

from paper_2511_02328_gb300 import synth


def test_noise_statistics_and_range():
    X = synth.filterbank(64, 1 << 15, seed=1)
    assert X.dtype == np.uint8 and X.shape == (64, 1 << 15)
    v = X.astype(np.float64)
    # a rounded N(128, 12) has variance 144 + 1/12
    assert abs(v.mean() - 128.0) < 0.02
    assert abs(v.std() - np.sqrt(144.0 + 1.0 / 12.0)) < 0.02
    # about 4.8e-7 of N(128, 12) lies beyond [-0.5, 255.5]: no clipping visible at this size
    assert v.min() > 60 and v.max() < 196


def test_deterministic_and_independent_of_chunking():
    a = synth.filterbank(37, 3000, seed=5)
    b = synth.filterbank(37, 3000, seed=5, rows_per_chunk=7)
    c = synth.filterbank(37, 3000, seed=6)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_rounding_half_to_even_and_clipping():
    # noise-free rows show the quantiser alone
    assert np.all(synth.filterbank(2, 8, seed=0, mean=128.5, sigma=0.0) == 128)
    assert np.all(synth.filterbank(2, 8, seed=0, mean=129.5, sigma=0.0) == 130)
    assert np.all(synth.filterbank(2, 8, seed=0, mean=300.0, sigma=0.0) == 255)
    assert np.all(synth.filterbank(2, 8, seed=0, mean=-7.0, sigma=0.0) == 0)


def test_pulse_amplitude_gives_the_requested_matched_filter_snr():
    # the pulse's excess summed over nchan x W samples, divided by the noise of
    # that sum (sigma * sqrt(nchan * W)), is the requested S/N
    for snr, nchan, W in [(15.0, 256, 10), (6.0, 4096, 3), (30.0, 1024, 200)]:
        a = synth.pulse_amplitude(snr, nchan, W)
        assert a * nchan * W / (12.0 * np.sqrt(nchan * W)) == pytest.approx(snr, rel=1e-12)
    assert synth.pulse_amplitude(15.0, 256, 10) == pytest.approx(15.0 * 12.0 / np.sqrt(2560.0), rel=1e-15)


def test_pulse_placement_with_clipped_edges():
    nchan, nsamp, W = 4, 50, 6
    offs = np.array([10, -3, 46, 60])          # interior, left edge, right edge, outside
    X = synth.filterbank(nchan, nsamp, seed=0, mean=100.0, sigma=0.0, pulses=[synth.Pulse(offs, W, 20.0)])
    ref = np.full((nchan, nsamp), 100, dtype=np.uint8)
    ref[0, 10:16] = 120
    ref[1, 0:3] = 120
    ref[2, 46:50] = 120
    assert np.array_equal(X, ref)
    # per-channel amplitudes
    X = synth.filterbank(2, 20, seed=0, mean=100.0, sigma=0.0,
                         pulses=[synth.Pulse(np.array([2, 5]), 3, np.array([4.0, 7.0]))])
    assert list(X[0, 2:5]) == [104] * 3 and list(X[1, 5:8]) == [107] * 3
    assert X.sum(dtype=np.int64) == 100 * 40 + 3 * 4 + 3 * 7


def test_rfi_shapes():
    nchan, nsamp = 16, 40000
    rfi = synth.RFI(narrow_channels=[3], bursts=[(100, 5, 50.0)], tones=[(8, 2000, 300, 0.01, 40.0)])
    X = synth.filterbank(nchan, nsamp, seed=2, rfi=rfi).astype(np.float64)
    quiet = np.ones(nsamp, dtype=bool)
    quiet[100:105] = False
    # persistent narrowband channel: mean + 3 sigma, variance x 2
    assert abs(X[3, quiet].mean() - (128.0 + 36.0)) < 0.3
    assert abs(X[3, quiet].std() - 12.0 * np.sqrt(2.0)) < 0.3
    # zero-DM burst: every channel raised by the amplitude for its 5 samples
    assert np.all(X[:, 100:105].mean(axis=0) > 128.0 + 40.0)
    # drifting tone: channel round(8 + 0.01 k) at sample 2000 + k
    for k in (0, 49, 50, 150, 299):
        c = int(round(8 + 0.01 * k))
        assert X[c, 2000 + k] > 128.0 + 40.0 - 5 * 12.0
    assert X[8, 2000:2050].mean() > 128.0 + 30.0 and X[9, 2000:2050].mean() < 140.0


def test_pulse_params_ranges_and_separation():
    tsamp = 49.152e-6
    pp = synth.pulse_params(20, 1002, (50.0, 1000.0), (0.2e-3, 10e-3), (6.0, 30.0),
                            (0.5, (262144 - 50000) * tsamp - 0.5), 0.45, tsamp)
    assert pp == synth.pulse_params(20, 1002, (50.0, 1000.0), (0.2e-3, 10e-3), (6.0, 30.0),
                                    (0.5, (262144 - 50000) * tsamp - 0.5), 0.45, tsamp)
    assert len(pp) == 20
    for p in pp:
        assert 50.0 <= p["dm"] <= 1000.0 and 6.0 <= p["snr"] <= 30.0
        assert max(1, round(0.2e-3 / tsamp)) <= p["width"] <= round(10e-3 / tsamp)
    # distinct slots of 0.45 s, jitter up to a quarter slot: neighbours >= 0.75 * 0.45 s apart
    t0 = np.array([p["t0"] for p in pp]) * tsamp
    assert np.all(np.diff(t0) >= 0.75 * 0.45 - 2 * tsamp)
    assert np.all(t0 >= 0.5 - tsamp) and np.all(t0 <= (262144 - 50000) * tsamp - 0.5 + tsamp)
    with pytest.raises(ValueError):
        synth.pulse_params(100, 0, (0, 1), (1e-3, 2e-3), (6, 7), (0.0, 1.0), 0.45, tsamp)
