"""Parity of the DM-time slice gridding (Sec. 2.4) with the oracle, through the
C ABI: the area path is bit-exact; the Lanczos-4 path (double on both sides,
different summation order) must agree except where the oracle's value before
rounding lies within 1e-9 of a half-integer, and then by at most one level."""
import numpy as np
import pytest

from oracle import grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _gpu_grid(Y, ns, M):
    from paper_2511_02328_gb300 import _lib
    ndm, nout = Y.shape
    S = -(-nout // ns)
    y = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.int32)).cuda()
    out = torch.empty((S, M, M), dtype=torch.uint8, device="cuda")
    work = torch.empty((S, 2), dtype=torch.int64, device="cuda")
    _lib.af_grid(y.data_ptr(), ndm, nout, ns, M, out.data_ptr(), work.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _lanczos_close(got, X, M):
    h, w = X.shape
    U = grid.lanczos4_matrix(h, M) @ X.astype(np.float64) @ grid.lanczos4_matrix(w, M).T
    lo, hi = U.min(), U.max()
    ref = grid.to_gray(U, (lo, hi)).astype(int)
    f = 255.0 * (U - lo) / (hi - lo + grid.EPS)
    tie = np.abs(f - np.floor(f) - 0.5) < 1e-9
    diff = got.astype(int) - ref
    assert np.all(np.abs(diff) <= 1)
    assert np.all(diff[~tie] == 0)


def test_area_slices_bit_exact():
    rng = np.random.default_rng(1)
    Y = rng.integers(0, 1 << 20, size=(1001, 25000), dtype=np.int32)
    Y[500, 7000:7010] += 1 << 24                     # a bright spot
    got = _gpu_grid(Y, 10000, 512)                  # slices 10000, 10000, 5000: all area
    assert got.shape == (3, 512, 512)
    ref = grid.grid(Y, 10000 * 1.0, 1.0, M=512)
    assert np.array_equal(got, ref)


def test_mixed_paths_and_ragged_last_slice():
    rng = np.random.default_rng(2)
    Y = rng.integers(0, 5000, size=(300, 4 * 900 + 77), dtype=np.int32)
    got = _gpu_grid(Y, 900, 128)                    # 4 area slices (300 > 128, 900 > 128), last 77 wide: Lanczos
    for s in range(4):
        assert np.array_equal(got[s], grid.grid_slice(Y[:, s * 900:(s + 1) * 900], M=128)[0]), s
    _lanczos_close(got[4], Y[:, 3600:], 128)


def test_lanczos_upsampling():
    rng = np.random.default_rng(3)
    Y = rng.integers(0, 1000, size=(40, 250), dtype=np.int32)
    got = _gpu_grid(Y, 100, 64)                     # 40 < 64: Lanczos on every slice
    for s in range(3):
        _lanczos_close(got[s], Y[:, s * 100:(s + 1) * 100], 64)


def test_constant_plane_and_single_column_slice():
    Y = np.full((600, 1001), 42, dtype=np.int32)
    got = _gpu_grid(Y, 500, 256)                    # last slice is one column wide
    assert got.shape == (3, 256, 256) and np.all(got == 0)


def test_search_plane_slices():
    # the 256-channel check plane (DM 0-500, pulse at DM 300) in 0.5 s slices:
    # 501 rows onto 256 (area) and onto 512 (Lanczos, the paper's M)
    from paper_2511_02328_gb300 import synth
    from paper_2511_02328_gb300.search import Plan
    import oracle
    from conftest import C1, dm_list
    cfg = C1
    offs = oracle.injection_offsets(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], 300.0, 8000)
    X = synth.filterbank(cfg["nchan"], cfg["nsamp"], seed=1,
                         pulses=[synth.Pulse(offs, 10, synth.pulse_amplitude(15.0, cfg["nchan"], 10))])
    p = Plan(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dm_list(cfg))
    plane = p.dedisperse(torch.from_numpy(X).cuda()).cpu().numpy()
    p.close()
    n_s, S, rng = grid.slices(plane.shape[1], 0.5, cfg["tsamp"])
    got = _gpu_grid(plane, n_s, 256)
    ref = grid.grid(plane, 0.5, cfg["tsamp"], M=256)
    assert np.array_equal(got, ref)
    got512 = _gpu_grid(plane, n_s, 512)
    for s, (c0, c1) in enumerate(rng):
        _lanczos_close(got512[s], plane[:, c0:c1], 512)
    # the slice holding the pulse has its brightest pixel near DM 300 (row 300/501 of the image)
    k = 8000 // n_s
    i, j = np.unravel_index(np.argmax(got[k]), got[k].shape)
    assert abs(i * 501 / 256 - 300) < 15


def test_argument_errors():
    from paper_2511_02328_gb300 import _lib
    y = torch.zeros((4, 10), dtype=torch.int32, device="cuda")
    o = torch.zeros(16, dtype=torch.uint8, device="cuda")
    for args in [(4, 10, 0, 4), (4, 10, 5, 1), (0, 10, 5, 4)]:
        with pytest.raises(_lib.AFError):
            _lib.af_grid(y.data_ptr(), args[0], args[1], args[2], args[3], o.data_ptr(), o.data_ptr())
