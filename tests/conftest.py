import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU-only oracle test")


@pytest.fixture(scope="session")
def small_lattice():
    """A 4^4 lattice with random links (eps 0.3), kappa 0.12, csw 1.0."""
    import synthetic
    L = (4, 4, 4, 4)
    U = synthetic.gauge_links(L, 0.3, 11)
    return dict(L=L, U=U, kappa=0.12, csw=1.0)
