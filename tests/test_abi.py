"""The C ABI library builds, loads and exports every symbol include/*.h
declares (no GPU needed; no compute calls)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-zA-Z_][\w\s\*]*?\b(af_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2511_02328_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["af_plan", "af_plan_destroy", "af_plan_delays", "af_plan_nout", "af_dedisperse",
              "af_boxcar_snr", "af_candidates", "af_search", "af_cluster", "af_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_2511_02328_gb300 import _lib
    missing = [n for n in sorted(_declared()) if n not in _lib.SIGNATURES]
    assert not missing, missing


def test_exports_are_c_symbols(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if " T " in l)
    for n in _declared():
        assert n in exported, n


def test_host_only_calls_without_gpu(libpath):
    from paper_2511_02328_gb300 import _lib
    assert "sm_103a" in _lib.af_version()
    # argument errors are reported before any CUDA call
    with pytest.raises(_lib.AFError) as e:
        _lib.af_plan(0, 1000.0, 1500.0, 1e-3, [0.0])
    assert e.value.code == _lib.AF_EINVAL
    with pytest.raises(_lib.AFError) as e:
        _lib.af_plan(16, 1000.0, 1500.0, 1e-3, [-5.0])
    assert e.value.code == _lib.AF_EINVAL
    assert "dm_list" in _lib.af_last_error()
    with pytest.raises(_lib.AFError) as e:
        _lib.af_diag_bounded_wait(0, 0)
    assert e.value.code == _lib.AF_EINVAL
    with pytest.raises(_lib.AFError) as e:
        _lib.af_diag_bounded_wait(0, (1 << 24) + 1)
    assert e.value.code == _lib.AF_EINVAL
