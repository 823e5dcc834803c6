import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


# Search configurations (sizes of the paper's workloads, Sec. 3 and Sec. 4).
C1 = dict(nchan=256, f_lo=1000.0, f_hi=1500.0, tsamp=98.304e-6, nsamp=1 << 15,
          dm_lo=0.0, dm_hi=500.0, dm_step=1.0, widths=[1, 2, 4, 8, 16, 32])
C2 = dict(nchan=4096, f_lo=1000.0, f_hi=1500.0, tsamp=49.152e-6, nsamp=1 << 18,
          dm_lo=0.0, dm_hi=1000.0, dm_step=1.0, widths=[1, 2, 4, 8, 16, 32, 64, 128, 256])


def dm_list(cfg):
    import numpy as np
    n = int(round((cfg["dm_hi"] - cfg["dm_lo"]) / cfg["dm_step"])) + 1
    return cfg["dm_lo"] + cfg["dm_step"] * np.arange(n, dtype=np.float64)


@pytest.fixture(scope="session")
def c1():
    return dict(C1)


@pytest.fixture(scope="session")
def c2():
    return dict(C2)
