"""The learned part end to end: chunks with pulses placed by the oracle's
injector and RFI, search, clustering, cut-outs, training on the GPU with the
library's kernels, and the comparison with the plain S/N threshold at equal
recall of injected pulses with S/N >= 8: the network must keep the recall
(within 1 %) while raising fewer false positives."""
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_network_beats_threshold_at_equal_recall():
    from paper_2511_02328_gb300 import _lib, classifier
    searcher = classifier.Searcher()
    c = classifier.CHUNK

    def offsets(dm, t0):
        return oracle.injection_offsets(c["nchan"], c["f_lo"], c["f_hi"], c["tsamp"], dm, t0)
    X, Y, _, _ = classifier.build_dataset(500, seed=1, searcher=searcher, offsets_fn=offsets)
    n_pos = int(Y.sum().item())
    assert X.shape[0] > 1000 and 0.2 < n_pos / X.shape[0] < 0.9
    model = _lib.af_model_create(128, 3)
    hist = classifier.train(model, X, Y, epochs=6, batch=128, lr=2e-3, seed=0)
    assert hist[-1] < hist[0]
    Xe, Ye, snr_e, rec_e = classifier.build_dataset(200, seed=99, searcher=searcher, offsets_fn=offsets)
    prob = classifier.predict(model, Xe, batch=128)
    res = classifier.evaluate(snr_e, prob, rec_e, nout=searcher.nout)
    print(res)
    assert res["injected"] > 300
    assert res["recall_cnn"] >= res["recall_threshold"] - 0.01
    assert res["fp_threshold"] > 0
    assert res["fp_cnn"] < 0.5 * res["fp_threshold"]
    _lib.af_model_destroy(model)
    searcher.close()
