import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")


@pytest.fixture(scope="session")
def sphere80():
    from synth import make_surface

    return make_surface(2)


@pytest.fixture(scope="session")
def sphere320():
    from synth import config_surface

    return config_surface("sphere320")


@pytest.fixture(scope="session")
def star_small():
    """Star surface r = 1 + 0.3 Re Y_6^3 at 180 elements (2,700 sources)."""
    from synth import make_surface, star_radius
    from synth.surfaces import STAR_Y63

    return make_surface(3, star_radius(STAR_Y63))


def rel_linf(a, b):
    """Normwise relative l-infinity error max|a-b| / max|b|."""
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b))))
