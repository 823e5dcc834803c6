"""The failure path of the bounded device waits.  The ring kernels wait on
mbarriers for at most a fixed number of polls; a wait that runs out raises the
error flag and the kernel returns, so a lost arrival becomes AF_ETIMEOUT on the
host instead of a hang.  Here that path is made to happen on a barrier that
nothing arrives at (af_diag_bounded_wait), the status is read back, and the
context is shown to be usable afterwards."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_wait_nothing_completes_times_out_and_the_context_stays_usable():
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import Plan
    rc, _ = _lib.af_diag_bounded_wait(1, 1024)                 # the arrival comes: no timeout
    assert rc == _lib.AF_OK
    rc, ms_small = _lib.af_diag_bounded_wait(0, 1024)          # nothing arrives
    assert rc == _lib.AF_ETIMEOUT and "ran out" in _lib.af_last_error()
    assert 0.0 < ms_small < 1000.0
    if ms_small < 10.0:                                        # more polls, a longer wait, still bounded
        rc, ms_big = _lib.af_diag_bounded_wait(0, 1 << 16)
        assert rc == _lib.AF_ETIMEOUT and ms_big > ms_small
        print("bounded wait: %.4f ms for 1024 polls, %.3f ms for 65536 polls (%.3f us per poll)"
              % (ms_small, ms_big, ms_big * 1e3 / 65536))
    rc, _ = _lib.af_diag_bounded_wait(1, 1 << 16)
    assert rc == _lib.AF_OK
    # the context is intact: a dedispersion after the timeouts is bit-exact
    nchan, f_lo, f_hi, tsamp = 32, 1000.0, 1500.0, 2e-4
    dms = np.arange(0.0, 40.0, 1.0)
    x = np.random.default_rng(5).integers(0, 256, (nchan, 4096), dtype=np.uint8)
    p = Plan(nchan, f_lo, f_hi, tsamp, dms)
    Y = p.dedisperse(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(Y, oracle.dedisperse(x, oracle.delay_table(nchan, f_lo, f_hi, tsamp, dms)))
    p.close()
