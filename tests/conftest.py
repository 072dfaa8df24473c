import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU-only test")


@pytest.fixture(scope="session")
def lossy_sphere():
    """Small lossy sphere r = 0.2, eps_r = 4 - 1j, pitch 1/16 (N = 1824), dense Z from the oracle."""
    import numpy as np

    import workloads as W
    from oracle.entries import Elements, zblock
    from oracle.mesh import build_mesh

    body = W.sphere(0.2, 4.0 - 1.0j, 1.0 / 16)
    mesh = build_mesh(body)
    E = Elements(mesh, W.K0)
    n = len(mesh["faces"])
    Z = zblock(E, np.arange(n), np.arange(n))
    return dict(body=body, mesh=mesh, E=E, Z=Z)
