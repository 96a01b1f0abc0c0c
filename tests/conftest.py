import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def small_oracle():
    """Oracle fit (Algorithm 2, FP64) of the N=8 workload, seed 0, with explicit restarts."""
    import oracle
    import synth

    w = synth.small_mixture(0)
    B0 = synth.restart_inits(w.M, w.N, w.N, 1000)
    res, Xw, V, mean = oracle.order_fit(w.X, w.M, w.N, w.iters, w.tol, B0, record=True)
    return w, B0, res, Xw, V, mean
