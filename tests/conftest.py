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


class SurfaceUnion:
    """Several surfaces discretized together (elements, sources and centers concatenated)."""

    def __init__(self, parts):
        self.parts = parts
        off = np.cumsum([0] + [p.n_elem for p in parts])
        self.n_elem = int(off[-1])
        cat = lambda k: np.concatenate([getattr(p, k) for p in parts], axis=-1)  # noqa: E731
        self.src_xyz, self.src_w, self.src_n = cat("src_xyz"), cat("src_w"), cat("src_n")
        self.ctr_xyz, self.ctr_r = cat("ctr_xyz"), cat("ctr_r")
        self.src_elem = np.concatenate([p.src_elem + o for p, o in zip(parts, off)]).astype(np.int32)
        self.ctr_elem = np.concatenate([p.ctr_elem + o for p, o in zip(parts, off)]).astype(np.int32)
        self.elem_eta = cat("elem_eta")
        nct = np.cumsum([0] + [p.n_ctr for p in parts])
        self.tgt_xyz = cat("tgt_xyz")
        self.tgt_ctr = np.concatenate([p.tgt_ctr + o for p, o in zip(parts, nct)]).astype(np.int32)


def two_spheres(meshes, gap, src_meshes=None):
    """Two unit spheres on the given flat meshes, the second shifted by 2 + gap along x; with
    src_meshes, sources from those (stage-2) meshes and centers from `meshes`."""
    from synth import surface_from_flat

    offs = [(0.0, 0.0, 0.0), (2.0 + gap, 0.0, 0.0)]
    if src_meshes is None:
        return SurfaceUnion([surface_from_flat(m, offset=o) for m, o in zip(meshes, offs)])
    return SurfaceUnion([surface_from_flat(m, offset=o, src_flat=m2) for m, m2, o in zip(meshes, src_meshes, offs)])
