"""Pins for the classifier and cut-out oracles: library routines (scipy
correlation, torch bfloat16 rounding), finite differences in float64, closed
forms (softmax cross-entropy, Adam's first step), and the geometry of a
dispersed pulse in the cut-outs."""
import numpy as np
import pytest

import oracle
from oracle import cnn, cutout
from paper_2511_02328_gb300 import synth


def test_bf16_round_matches_library():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 10, 10000).astype(np.float32),
                        np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8, 0.0, 65504.0], dtype=np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(cutout.bf16_round(x), ref)
    assert cutout.bf16_round(np.float32(1 + 2 ** -8)) == 1.0            # tie to even
    assert cutout.bf16_round(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6


def test_conv3x3_matches_scipy():
    from scipy.signal import correlate2d
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 9, 7, 3))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = cnn.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[n, :, :, i], w[o, :, :, i], mode="same") for i in range(3))
            assert np.allclose(y[n, :, :, o], ref)


def test_maxpool_ties_and_routing():
    x = np.array([[[[1.0], [3.0]], [[3.0], [0.0]]]])  # 1 x 2 x 2 x 1, tie between (0,1) and (1,0)
    y, idx = cnn.maxpool2(x)
    assert y[0, 0, 0, 0] == 3.0 and idx[0, 0, 0, 0] == 1
    g = cnn.maxpool2_grad(np.ones((1, 1, 1, 1)), idx, x.shape)
    assert g[0, 0, 1, 0] == 1.0 and g.sum() == 1.0


def test_softmax_ce_gradient_closed_form():
    logits = np.array([[2.0, -1.0], [0.5, 0.25]])
    y = np.array([0, 1])
    loss, d, pr = cnn.softmax_ce(logits, y)
    onehot = np.eye(2)[y]
    assert np.allclose(d, (pr - onehot) / 2)
    assert np.isclose(loss, -np.mean(np.log(pr[[0, 1], [0, 1]])))


def test_network_gradients_by_finite_differences():
    rng = np.random.default_rng(3)
    p = {k: v.astype(np.float64) for k, v in cnn.init_params(5).items()}
    for l in range(3):
        p["b%d" % l] = rng.normal(0, 0.1, p["b%d" % l].shape)
    x = rng.uniform(0, 1, (2, 64, 64, 2))
    y = np.array([0, 1])
    loss, _, g = cnn.loss_and_grads(p, x, y, bf16=False)
    eps = 1e-6
    checks = [("w0", (3, 1, 2, 1)), ("w1", (5, 0, 0, 7)), ("w2", (60, 2, 1, 31)), ("b1", (4,)), ("fw", (1, 17)),
              ("fb", (0,))]
    for k, ix in checks:
        q = {kk: vv.copy() for kk, vv in p.items()}
        q[k][ix] += eps
        lp = cnn.loss_and_grads(q, x, y, bf16=False)[0]
        q[k][ix] -= 2 * eps
        lm = cnn.loss_and_grads(q, x, y, bf16=False)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[k][ix]) <= 1e-6 + 1e-4 * abs(fd), (k, ix, fd, g[k][ix])
    for ix in [(0, 10, 11, 0), (1, 40, 3, 1)]:
        xx = x.copy()
        xx[ix] += eps
        lp = cnn.loss_and_grads(p, xx, y, bf16=False)[0]
        xx[ix] -= 2 * eps
        lm = cnn.loss_and_grads(p, xx, y, bf16=False)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g["x"][ix]) <= 1e-7 + 1e-4 * abs(fd)


def test_adam_first_step_closed_form():
    p = {"a": np.array([1.0, -2.0], dtype=np.float32)}
    g = {"a": np.array([0.5, -3.0], dtype=np.float32)}
    out = cnn.adam_step(p, g, {}, lr=0.01)
    # first step: m_hat = g, v_hat = g^2 -> update lr * g / (|g| + eps)
    assert np.allclose(out["a"], [1.0 - 0.01, -2.0 + 0.01], atol=1e-6)


def test_cutout_small_example_by_hand():
    plane = np.arange(5 * 200, dtype=np.int32).reshape(5, 200)
    got = cutout.dm_time(plane, d=2, t=100, w=4)           # b = 2, bins start at 100 - 64
    # plane rows 0..4 map to cut-out rows i = 30..34; the other rows are zero
    assert got[29].sum() == 0 and got[35].sum() == 0 and got[30].sum() > 0
    r = plane[2].astype(np.int64)
    assert got[32, 0] == r[36] + r[37] and got[32, 63] == r[162] + r[163]
    assert got[31, 10] == plane[1, 56] + plane[1, 57]
    # bins before the start of the row are zero
    edge = cutout.dm_time(plane, d=0, t=10, w=1)            # b = 1, bins start at -22
    assert edge[32, 21] == 0 and edge[32, 22] == plane[0, 0]


def test_cutout_normalisation_range_and_constant():
    v = cutout._normalise(np.array([[5, 5], [5, 5]]))
    assert np.all(v == 0.0)
    v = cutout._normalise(np.array([[3, 7], [11, 3]]))
    assert v.min() == 0.0 and abs(v.max() - 1.0) < 1e-2


def test_dispersed_pulse_is_vertical_at_its_dm():
    nchan, f_lo, f_hi, tsamp, nsamp = 256, 1000.0, 1500.0, 98.304e-6, 1 << 14
    dms = np.arange(0.0, 120.0, 1.0)
    t0, dm0, W = 6000, 80.0, 6
    offs = oracle.injection_offsets(nchan, f_lo, f_hi, tsamp, dm0, t0)
    X = synth.filterbank(nchan, nsamp, seed=9, pulses=[synth.Pulse(offs, W, synth.pulse_amplitude(60.0, nchan, W))])
    D = oracle.delay_table(nchan, f_lo, f_hi, tsamp, dms)
    Y = oracle.dedisperse(X, D)
    ft = cutout.freq_time(X, D, 80, t0, W, Y.shape[1])
    peak_bins = ft.argmax(axis=1)
    assert np.all(np.abs(peak_bins - 32) <= 3)              # every channel group peaks at the pulse
    ft_wrong = cutout.freq_time(X, D, 40, t0, W, Y.shape[1])
    assert np.ptp(ft_wrong.argmax(axis=1)) > 10             # at DM 40 the sweep remains
    dt = cutout.dm_time(Y, 80, t0, W)
    i, j = np.unravel_index(dt.argmax(), dt.shape)
    assert abs(i - 32) <= 2 and abs(j - 32) <= 3
    c = cutout.cutouts(X, D, Y, [(80, t0, W)])
    assert c.shape == (1, 2, 64, 64) and c.min() >= 0 and c.max() <= 1
