import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def hex_sphere():
    """Hex 32^3 unit cube, vapour sphere R=0.25 at the centre; alpha from 8^3 midpoint samples."""
    import synth
    m = synth.hex_box(32)
    reg = dict(type="spheres", spheres=[(0.5, 0.5, 0.5, 0.25)])
    a = synth.alpha(m, reg, mode="hexgrid", level=3)
    T, Tb = synth.temperature(m, reg, dict(kind="radial", dT=5.0))
    return m, reg, a, T, Tb
