import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


_CACHE = {}


def make_matrix(name_or_workload):
    """Cached (workload, row_ptr, col, val) for a named or given workload."""
    import workloads as W
    w = W.config(name_or_workload) if isinstance(name_or_workload, str) else name_or_workload
    key = (tuple(w.level_sizes), w.nnz_per_row, w.seed, w.sigma)
    if key not in _CACHE:
        _CACHE[key] = W.generate(w)
    rp, c, v = _CACHE[key]
    return w, rp, c, v


@pytest.fixture(scope="session")
def small_matrix():
    return make_matrix("small")


@pytest.fixture(scope="session")
def c1_matrix():
    return make_matrix("c1")


def dense(rp, c, v, n=None):
    n = rp.shape[0] - 1 if n is None else n
    A = np.zeros((rp.shape[0] - 1, n))
    for i in range(rp.shape[0] - 1):
        A[i, c[rp[i]:rp[i + 1]]] += v[rp[i]:rp[i + 1]]
    return A
