"""The classifier on the GPU against the oracle: the tcgen05 tensor-core GEMM
in all four operand layouts, cut-outs (bit-exact bf16), forward logits (rel
1e-2) on both inference paths (the fused mma.sync kernel for small batches,
the tcgen05 implicit-GEMM layers for large ones), gradients of the tcgen05
training path (cosine >= 0.999 and rel-L2 <= 2e-2 per tensor) at two batch
sizes, Adam, training that lowers the loss, checkpoint round trip, and
af_classify."""
import numpy as np
import pytest

import oracle
from oracle import cnn, cutout
from paper_2511_02328_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _bf16_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()


def _flat(p):
    return np.concatenate([p["w0"].ravel(), p["b0"], p["w1"].ravel(), p["b1"], p["w2"].ravel(), p["b2"],
                           p["fw"].ravel(), p["fb"]]).astype(np.float32)


def _unflat(v):
    shapes = [("w0", (16, 3, 3, 2)), ("b0", (16,)), ("w1", (32, 3, 3, 16)), ("b1", (32,)), ("w2", (64, 3, 3, 32)),
              ("b2", (64,)), ("fw", (2, 64)), ("fb", (2,))]
    out, o = {}, 0
    for k, s in shapes:
        n = int(np.prod(s))
        out[k] = v[o:o + n].reshape(s)
        o += n
    return out


@pytest.mark.parametrize("layout", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(200, 48, 96), (64, 16, 32), (1000, 64, 288), (37, 40, 24)])
def test_gemm_layouts(layout, shape):
    from paper_2511_02328_gb300 import _lib
    M, N, K = shape
    rng = np.random.default_rng(M + N + K + layout)
    A = cutout.bf16_round(rng.normal(size=(M, K)).astype(np.float32))
    B = cutout.bf16_round(rng.normal(size=(K, N)).astype(np.float32))
    ref = A.astype(np.float64) @ B.astype(np.float64)
    a_store = A if layout in (0, 1) else A.T
    b_store = B.T if layout in (0, 3) else B
    da, db = _bf16_dev(a_store), _bf16_dev(b_store)
    lda, ldb = a_store.shape[1], b_store.shape[1]
    if lda % 8 or ldb % 8:
        pytest.skip("pitch not a multiple of 8")
    c = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    _lib.af_nn_gemm(layout, 0, da.data_ptr(), lda, db.data_ptr(), ldb, M, N, K, 1, c.data_ptr(), N)
    torch.cuda.synchronize()
    got = c.cpu().numpy()
    assert np.allclose(got, ref, rtol=1e-4, atol=1e-3 * np.sqrt(K))
    # split-K atomic accumulation and the bias + ReLU epilogue
    c.zero_()
    _lib.af_nn_gemm(layout, 2, da.data_ptr(), lda, db.data_ptr(), ldb, M, N, K, 3, c.data_ptr(), N)
    bias = torch.from_numpy(rng.normal(size=N).astype(np.float32)).cuda()
    c2 = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    _lib.af_nn_gemm(layout, 1, da.data_ptr(), lda, db.data_ptr(), ldb, M, N, K, 1, c2.data_ptr(), N, bias.data_ptr())
    torch.cuda.synchronize()
    assert np.allclose(c.cpu().numpy(), ref, rtol=1e-4, atol=1e-3 * np.sqrt(K))
    assert np.allclose(c2.cpu().numpy(), np.maximum(ref + bias.cpu().numpy(), 0), rtol=1e-4, atol=1e-3 * np.sqrt(K))


@pytest.fixture(scope="module")
def pulse_data():
    nchan, f_lo, f_hi, tsamp, nsamp = 256, 1000.0, 1500.0, 98.304e-6, 1 << 14
    dms = np.arange(0.0, 120.0, 1.0)
    t0, dm0, W = 6000, 80.0, 6
    offs = oracle.injection_offsets(nchan, f_lo, f_hi, tsamp, dm0, t0)
    X = synth.filterbank(nchan, nsamp, seed=9, pulses=[synth.Pulse(offs, W, synth.pulse_amplitude(40.0, nchan, W))])
    D = oracle.delay_table(nchan, f_lo, f_hi, tsamp, dms)
    Y = oracle.dedisperse(X, D)
    cands = [(80, t0, W), (3, 100, 1), (117, 12000, 32), (50, Y.shape[1] - 5, 256), (0, 0, 2)]
    return dict(nchan=nchan, f_lo=f_lo, f_hi=f_hi, tsamp=tsamp, dms=dms, X=X, D=D, Y=Y, cands=cands)


def _cand_array(cands):
    from paper_2511_02328_gb300 import _lib
    a = np.zeros(len(cands), dtype=_lib.CAND_DTYPE)
    for i, (d, t, w) in enumerate(cands):
        a[i] = (d, t, w, 0.0, t)
    return torch.from_numpy(a.view(np.uint8)).cuda()


def test_cutouts_bit_exact(pulse_data):
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import Plan
    s = pulse_data
    p = Plan(s["nchan"], s["f_lo"], s["f_hi"], s["tsamp"], s["dms"])
    xd = torch.from_numpy(s["X"]).cuda()
    plane = p.dedisperse(xd)
    cd = _cand_array(s["cands"])
    n = len(s["cands"])
    out = torch.empty((n, 64, 64, 2), dtype=torch.bfloat16, device="cuda")
    _lib.af_cutouts(p.handle, xd.data_ptr(), s["X"].shape[1], plane.data_ptr(), plane.shape[1], cd.data_ptr(), n,
                    out.data_ptr())
    torch.cuda.synchronize()
    got = out.float().cpu().numpy().transpose(0, 3, 1, 2)
    ref = cutout.cutouts(s["X"], s["D"], s["Y"], s["cands"])
    assert np.array_equal(got, ref)
    p.close()


@pytest.mark.parametrize("nsamp", [1 << 13, (1 << 13) + 5])
def test_cutouts_wide_band_and_foreign_rows(nsamp):
    """1024 channels (16 per frequency-time row, 128 per CTA of the cluster),
    wide and narrow bins at both ends of the plane, and candidates whose DM
    index is not a row of the plan (zero cut-outs, the rest unaffected); input
    rows of whole 16-byte blocks (16-byte loads) and not (byte loads)."""
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import Plan
    nchan, f_lo, f_hi, tsamp = 1024, 1200.0, 1500.0, 1e-4
    dms = np.arange(0.0, 40.0, 1.0)
    X = synth.filterbank(nchan, nsamp, seed=21)
    D = oracle.delay_table(nchan, f_lo, f_hi, tsamp, dms)
    Y = oracle.dedisperse(X, D)
    nout = Y.shape[1]
    good = [(20, nout // 2, 64), (0, 3, 1), (39, nout - 1, 16), (5, 900, 128)]
    cands = good[:2] + [(-1, 100, 4)] + good[2:] + [(len(dms), 50, 8)]
    p = Plan(nchan, f_lo, f_hi, tsamp, dms)
    xd = torch.from_numpy(X).cuda()
    plane = p.dedisperse(xd)
    cd = _cand_array(cands)
    out = torch.empty((len(cands), 64, 64, 2), dtype=torch.bfloat16, device="cuda")
    _lib.af_cutouts(p.handle, xd.data_ptr(), nsamp, plane.data_ptr(), nout, cd.data_ptr(), len(cands),
                    out.data_ptr())
    torch.cuda.synchronize()
    got = out.float().cpu().numpy().transpose(0, 3, 1, 2)
    ref = cutout.cutouts(X, D, Y, good)
    assert np.array_equal(got[[0, 1, 3, 4]], ref)
    assert not got[2].any() and not got[5].any()
    p.close()


def test_forward_and_gradients_match_oracle():
    from paper_2511_02328_gb300 import _lib
    rng = np.random.default_rng(7)
    p = cnn.init_params(3)
    for l in range(3):
        p["b%d" % l] = rng.normal(0, 0.05, p["b%d" % l].shape).astype(np.float32)
    n = 24
    x = cutout.bf16_round(rng.uniform(0, 1, (n, 64, 64, 2)).astype(np.float32))
    y = rng.integers(0, 2, n).astype(np.int32)
    m = _lib.af_model_create(64, 1)
    assert _lib.af_model_nparams(m) == _lib.NPARAMS
    _lib.af_model_set_params(m, _flat(p))
    xd = _bf16_dev(x)
    yd = torch.from_numpy(y).cuda()
    logits = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    prob = torch.empty(n, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    _lib.af_model_forward(m, xd.data_ptr(), n, logits.data_ptr(), prob.data_ptr())
    _lib.af_model_backward(m, xd.data_ptr(), yd.data_ptr(), n, loss.data_ptr())
    torch.cuda.synchronize()
    ref_loss, ref_logits, ref_g = cnn.loss_and_grads(p, x, y, bf16=True)
    lg = logits.cpu().numpy()
    assert np.max(np.abs(lg - ref_logits)) <= 1e-2 * max(1.0, np.abs(ref_logits).max())
    e = np.exp(ref_logits - ref_logits.max(1, keepdims=True))
    assert np.allclose(prob.cpu().numpy(), e[:, 1] / e.sum(1), atol=5e-3)
    assert abs(float(loss.item()) - ref_loss) <= 1e-2 * max(1.0, ref_loss)
    g = _unflat(_lib.af_model_get_grads(m))
    for k in ["w0", "b0", "w1", "b1", "w2", "b2", "fw", "fb"]:
        a, b = g[k].astype(np.float64).ravel(), np.asarray(ref_g[k], dtype=np.float64).ravel()
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30)
        rel = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-30)
        assert cos >= 0.999 and rel <= 2e-2, (k, cos, rel)
    _lib.af_model_destroy(m)


def _model_with(params, max_batch, umma_min, monkeypatch):
    from paper_2511_02328_gb300 import _lib
    monkeypatch.setenv("AFGB_CNN_UMMA_MIN", str(umma_min))
    m = _lib.af_model_create(max_batch, 1)
    _lib.af_model_set_params(m, _flat(params))
    return m


def test_inference_paths_match_oracle_and_each_other(monkeypatch):
    """A batch of 96 through the tcgen05 layers (conv + bias + ReLU + pool in
    one kernel per layer) and through the fused mma.sync kernel: both within
    the logit tolerance of the oracle, P(pulse) of the two within 5e-3."""
    from paper_2511_02328_gb300 import _lib
    rng = np.random.default_rng(17)
    p = cnn.init_params(5)
    for l in range(3):
        p["b%d" % l] = rng.normal(0, 0.05, p["b%d" % l].shape).astype(np.float32)
    n = 96
    x = cutout.bf16_round(rng.uniform(0, 1, (n, 64, 64, 2)).astype(np.float32))
    x[:8] = 0.0                                         # all-zero images: ReLU ties in every pool window
    ref_logits = cnn.forward(p, x, bf16=True)[0]
    xd = _bf16_dev(x)
    out = {}
    for name, umma_min in (("tcgen05", 1), ("fused", 1 << 20)):
        m = _model_with(p, n, umma_min, monkeypatch)
        logits = torch.empty((n, 2), dtype=torch.float32, device="cuda")
        prob = torch.empty(n, dtype=torch.float32, device="cuda")
        _lib.af_model_forward(m, xd.data_ptr(), n, logits.data_ptr(), prob.data_ptr())
        torch.cuda.synchronize()
        lg = logits.cpu().numpy()
        assert np.max(np.abs(lg - ref_logits)) <= 1e-2 * max(1.0, np.abs(ref_logits).max()), name
        out[name] = prob.cpu().numpy()
        _lib.af_model_get_params(m)                      # reports a bounded wait that ran out
        _lib.af_model_destroy(m)
    assert np.max(np.abs(out["tcgen05"] - out["fused"])) <= 5e-3


def test_gradients_match_oracle_larger_batch(monkeypatch):
    """Gradients of the tcgen05 training path on 72 images (several weight-
    gradient pixel runs per layer, the split-K atomics), against the oracle."""
    from paper_2511_02328_gb300 import _lib
    rng = np.random.default_rng(29)
    p = cnn.init_params(9)
    for l in range(3):
        p["b%d" % l] = rng.normal(0, 0.05, p["b%d" % l].shape).astype(np.float32)
    n = 72
    x = cutout.bf16_round(rng.uniform(0, 1, (n, 64, 64, 2)).astype(np.float32))
    y = rng.integers(0, 2, n).astype(np.int32)
    m = _model_with(p, n, 1, monkeypatch)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    _lib.af_model_backward(m, _bf16_dev(x).data_ptr(), torch.from_numpy(y).cuda().data_ptr(), n, loss.data_ptr())
    torch.cuda.synchronize()
    ref_loss, _, ref_g = cnn.loss_and_grads(p, x, y, bf16=True)
    assert abs(float(loss.item()) - ref_loss) <= 1e-2 * max(1.0, ref_loss)
    g = _unflat(_lib.af_model_get_grads(m))
    for k in ["w0", "b0", "w1", "b1", "w2", "b2", "fw", "fb"]:
        a, b = g[k].astype(np.float64).ravel(), np.asarray(ref_g[k], dtype=np.float64).ravel()
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30)
        rel = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-30)
        assert cos >= 0.999 and rel <= 2e-2, (k, cos, rel)
    _lib.af_model_destroy(m)


@pytest.mark.parametrize("n", [1, 3])
def test_gradients_match_oracle_tiny_batches(n, monkeypatch):
    """Gradients of the tcgen05 training path on 1 and 3 images (fewer tiles
    than thread blocks: the first layer's in-kernel pool backward with one of
    its two warp groups idle, the second layer's weight gradient on a single
    tile per block), one all-zero image among them, against the oracle."""
    from paper_2511_02328_gb300 import _lib
    rng = np.random.default_rng(41 + n)
    p = cnn.init_params(11)
    for l in range(3):
        p["b%d" % l] = rng.normal(0, 0.05, p["b%d" % l].shape).astype(np.float32)
    x = cutout.bf16_round(rng.uniform(0, 1, (n, 64, 64, 2)).astype(np.float32))
    if n > 1:
        x[1] = 0.0
    y = (np.arange(n) % 2).astype(np.int32)
    m = _model_with(p, 4, 1, monkeypatch)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    _lib.af_model_backward(m, _bf16_dev(x).data_ptr(), torch.from_numpy(y).cuda().data_ptr(), n, loss.data_ptr())
    torch.cuda.synchronize()
    ref_loss, _, ref_g = cnn.loss_and_grads(p, x, y, bf16=True)
    assert abs(float(loss.item()) - ref_loss) <= 1e-2 * max(1.0, ref_loss)
    g = _unflat(_lib.af_model_get_grads(m))
    for k in ["w0", "b0", "w1", "b1", "w2", "b2", "fw"]:
        a, b = g[k].astype(np.float64).ravel(), np.asarray(ref_g[k], dtype=np.float64).ravel()
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30)
        rel = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-30)
        assert cos >= 0.999 and rel <= 2e-2, (k, cos, rel)
    # dL/dfb = the batch mean of P - onehot: on a few images it can be near 0,
    # so it is held to the probabilities' own tolerance (5e-3), absolutely
    assert np.max(np.abs(g["fb"].astype(np.float64) - np.asarray(ref_g["fb"], dtype=np.float64))) <= 5e-3
    _lib.af_model_get_params(m)                          # reports a bounded wait that ran out
    _lib.af_model_destroy(m)


def test_adam_and_training_lower_the_loss(tmp_path):
    from paper_2511_02328_gb300 import _lib
    rng = np.random.default_rng(11)
    n = 64
    # separable toy task: bright centre stripe (class 1) vs noise (class 0)
    x = rng.uniform(0, 0.5, (n, 64, 64, 2)).astype(np.float32)
    y = (rng.uniform(size=n) < 0.5).astype(np.int32)
    x[y == 1, 28:36, :, :] += 0.5
    x = cutout.bf16_round(x)
    m = _lib.af_model_create(n, 5)
    p0 = _lib.af_model_get_params(m)
    xd, yd = _bf16_dev(x), torch.from_numpy(y).cuda()
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    # one step equals the oracle's Adam step on the GPU's own gradients
    _lib.af_model_backward(m, xd.data_ptr(), yd.data_ptr(), n, loss.data_ptr())
    g = _lib.af_model_get_grads(m)
    _lib.af_train_step(m, xd.data_ptr(), yd.data_ptr(), n, 1e-3, loss.data_ptr())
    torch.cuda.synchronize()
    p1 = _lib.af_model_get_params(m)
    ref = cnn.adam_step({"a": p0.copy()}, {"a": g}, {}, lr=1e-3)["a"]
    assert np.allclose(p1, ref, atol=1e-6)
    first = float(loss.item())
    for _ in range(60):
        _lib.af_train_step(m, xd.data_ptr(), yd.data_ptr(), n, 3e-3, loss.data_ptr())
    torch.cuda.synchronize()
    assert float(loss.item()) < 0.5 * first
    path = tmp_path / "cnn.ckpt"
    _lib.af_model_save(m, path)
    m2 = _lib.af_model_create(n, 0)
    _lib.af_model_load(m2, path)
    assert np.array_equal(_lib.af_model_get_params(m2), _lib.af_model_get_params(m))
    _lib.af_model_destroy(m)
    _lib.af_model_destroy(m2)


def test_classify_equals_cutouts_then_forward(pulse_data):
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import Plan
    s = pulse_data
    p = Plan(s["nchan"], s["f_lo"], s["f_hi"], s["tsamp"], s["dms"])
    xd = torch.from_numpy(s["X"]).cuda()
    plane = p.dedisperse(xd)
    cd = _cand_array(s["cands"])
    n = len(s["cands"])
    m = _lib.af_model_create(2, 4)          # batch smaller than n: classify works in pieces
    prob = torch.empty(n, dtype=torch.float32, device="cuda")
    _lib.af_classify(m, p.handle, xd.data_ptr(), s["X"].shape[1], plane.data_ptr(), plane.shape[1], cd.data_ptr(),
                     n, prob.data_ptr())
    cut = torch.empty((n, 64, 64, 2), dtype=torch.bfloat16, device="cuda")
    _lib.af_cutouts(p.handle, xd.data_ptr(), s["X"].shape[1], plane.data_ptr(), plane.shape[1], cd.data_ptr(), n,
                    cut.data_ptr())
    prob2 = torch.empty(n, dtype=torch.float32, device="cuda")
    for i0 in range(0, n, 2):
        k = min(2, n - i0)
        _lib.af_model_forward(m, cut[i0:].data_ptr(), k, 0, prob2[i0:].data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(prob, prob2)
    _lib.af_model_destroy(m)
    p.close()
