"""af_boxcar_snr_noalloc: the boxcar S/N call for callers that cannot call
cudaMalloc (a real-time receiver thread that must not stall on an allocation,
or an application whose memory pool owns the whole GPU).  It must give the
same S/N and best widths as af_boxcar_snr, call after call, although its
scratch is one static device array reused by every call.

This file is named to be collected last, so that a run stopping at its first
failure has already run every other test."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _plane_and_reference(seed, nchan, nsamp, dms, widths):
    from paper_2511_02328_gb300.search import Plan
    rng = np.random.default_rng(seed)
    x = torch.from_numpy(rng.integers(0, 256, (nchan, nsamp), dtype=np.uint8)).cuda()
    p = Plan(nchan, 1000.0, 1500.0, 1e-4, dms)
    plane = p.dedisperse(x)
    snr, bw = p.boxcar_snr(plane, widths)          # the existing entry point, plan scratch
    torch.cuda.synchronize()
    ref = (snr.cpu().numpy(), bw.cpu().numpy())
    p.close()
    return plane, ref


def test_noalloc_matches_boxcar_snr_two_calls_in_a_row():
    from paper_2511_02328_gb300 import _lib
    cases = [(11, 96, 20000, np.arange(0, 64, 1.0), [1, 2, 4, 8, 16]),
             (12, 33, 9000, np.arange(0, 17, 0.5), [1, 3, 32])]   # different shape, stale scratch behind it
    for seed, nchan, nsamp, dms, widths in cases:
        plane, (ref_snr, ref_bw) = _plane_and_reference(seed, nchan, nsamp, dms, widths)
        ndm, nout = plane.shape
        snr = torch.full((ndm, nout), np.nan, dtype=torch.float32, device="cuda")
        bw = torch.full((ndm, nout), 77, dtype=torch.uint8, device="cuda")
        _lib.af_boxcar_snr_noalloc(plane.data_ptr(), ndm, nout, nchan, widths, snr.data_ptr(), bw.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = snr.cpu().numpy().astype(np.float64)
        fin = np.isfinite(ref_snr)
        assert np.array_equal(np.isfinite(got), fin)
        err = np.abs(got[fin] - ref_snr[fin]) / np.maximum(1.0, np.abs(ref_snr[fin]))
        assert float(err.max()) <= TOL
        assert np.array_equal(bw.cpu().numpy(), ref_bw)
        # and, independently of the plan path, the oracle's S/N of the same plane
        o_snr, _ = oracle.boxcar_snr(plane.cpu().numpy(), widths)
        ofin = np.isfinite(o_snr)
        assert np.array_equal(np.isfinite(got), ofin)
        oerr = np.abs(got[ofin] - o_snr[ofin]) / np.maximum(1.0, np.abs(o_snr[ofin]))
        assert float(oerr.max()) <= TOL


def test_noalloc_at_its_row_limit_without_width_output():
    """AF_NOALLOC_MAX_ROWS rows (the last row's constants at the end of the
    static array), no best-width output, against the oracle and against
    af_boxcar_snr; then a one-row call behind it on the same scratch."""
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import Plan
    ndm, nout, nchan = _lib.AF_NOALLOC_MAX_ROWS, 300, 16
    widths = [1, 2, 4, 8, 16, 32]
    rng = np.random.default_rng(21)
    Y = rng.integers(0, 255 * nchan + 1, (ndm, nout)).astype(np.int32)
    Y[-1, 100:110] = 255 * nchan                       # a pulse in the last row
    plane = torch.from_numpy(Y).cuda()
    snr = torch.full((ndm, nout), np.nan, dtype=torch.float32, device="cuda")
    _lib.af_boxcar_snr_noalloc(plane.data_ptr(), ndm, nout, nchan, widths, snr.data_ptr(), 0,
                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = snr.cpu().numpy().astype(np.float64)
    o_snr, _ = oracle.boxcar_snr(Y, widths)
    fin = np.isfinite(o_snr)
    assert np.array_equal(np.isfinite(got), fin)
    err = np.abs(got[fin] - o_snr[fin]) / np.maximum(1.0, np.abs(o_snr[fin]))
    assert float(err.max()) <= TOL
    p = Plan(nchan, 1000.0, 1500.0, 1e-4, np.linspace(0.0, 1.0, ndm))
    ref, _ = p.boxcar_snr(plane, widths)
    torch.cuda.synchronize()
    assert np.array_equal(np.isfinite(ref.cpu().numpy()), fin)
    assert float(np.max(np.abs(ref.cpu().numpy()[fin] - got[fin]) / np.maximum(1.0, np.abs(got[fin])))) <= TOL
    p.close()
    one = torch.full((1, nout), np.nan, dtype=torch.float32, device="cuda")
    _lib.af_boxcar_snr_noalloc(plane[-1:].data_ptr(), 1, nout, nchan, widths, one.data_ptr(), 0,
                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    g1, r1 = one.cpu().numpy()[0].astype(np.float64)[fin[-1]], o_snr[-1][fin[-1]]
    assert float(np.max(np.abs(g1 - r1) / np.maximum(1.0, np.abs(r1)))) <= TOL


def test_noalloc_rejects_more_rows_than_its_scratch():
    from paper_2511_02328_gb300 import _lib
    plane = torch.zeros((1, 64), dtype=torch.int32, device="cuda")
    snr = torch.empty((1, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(_lib.AFError) as e:
        _lib.af_boxcar_snr_noalloc(plane.data_ptr(), _lib.AF_NOALLOC_MAX_ROWS + 1, 64, 16, [1], snr.data_ptr())
    assert e.value.code == _lib.AF_EINVAL
    assert "static scratch" in _lib.af_last_error()
