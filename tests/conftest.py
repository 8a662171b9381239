import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def exp2d_case():
    """The small 2D case: n=4096 uniform points, exp(-r/0.2)+1e-2 I, SVD leaves, eps=1e-6."""
    import synth
    from oracle import hmatrix as hm
    p = synth.exp2d_problem(4096, seed=0)
    H = hm.build_hmatrix(p, 1e-6, leaf_size=64, eta=2.0, method="svd")
    C = hm.compress(H)
    return p, H, C


@pytest.fixture(scope="session")
def matern_small_case():
    """A 3D Matern case built with ACA + recompression: n=3000, eps=1e-6."""
    import synth
    from oracle import hmatrix as hm
    p = synth.matern_problem(3000, seed=100)
    H = hm.build_hmatrix(p, 1e-6, leaf_size=64, eta=2.0, method="aca")
    C = hm.compress(H)
    return p, H, C
