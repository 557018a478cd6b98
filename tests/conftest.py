import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def read_golden(name):
    """Numeric rows of a golden fixture (comment lines start with '#')."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


@pytest.fixture
def golden():
    return read_golden


def df32_pack(x):
    """float64 [state][b] values as the library's double-float vectors (float32 numpy array):
    hi = rn32(x), lo = rn32(x - hi). For b = 4 each state holds (hi_0, hi_1, lo_0, lo_1, hi_2, hi_3,
    lo_2, lo_3), shape [state][8]; other b hold (hi, lo) per element, shape [state][b][2]."""
    import numpy as np
    x = np.asarray(x, dtype=np.float64)
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    if x.ndim == 2 and x.shape[1] == 4:
        out = np.empty((x.shape[0], 2, 2, 2), np.float32)        # [state][pair][hi, lo][lane]
        out[:, :, 0, :] = hi.reshape(-1, 2, 2)
        out[:, :, 1, :] = lo.reshape(-1, 2, 2)
        return out.reshape(x.shape[0], 8)
    out = np.empty(x.shape + (2,), np.float32)
    out[..., 0], out[..., 1] = hi, lo
    return out


def df32_unpack(a, b):
    """The float64 values (hi + lo) of library double-float vectors laid out as df32_pack makes them."""
    import numpy as np
    a = np.asarray(a, dtype=np.float64)
    if b == 4:
        v = a.reshape(a.shape[0], 2, 2, 2)
        return (v[:, :, 0, :] + v[:, :, 1, :]).reshape(a.shape[0], 4)
    return a[..., 0] + a[..., 1]
