"""Pins of the urchin geometry and its adaptive meshing (Section 6.1), no GPU.

* The conical rule behind the resolution measure is exact to total degree 2n - 1 on the triangle
  (integrals a! b! / (a + b + 2)!) and not beyond; the basis it builds is orthonormal and hierarchical.
* The measure is zero for maps of degree <= 2, equals the size of the cubic and quartic parts of a
  map built from them, and on a sphere falls by about 2^3 per bisection (a smooth map's cubic
  coefficients scale with the element size cubed).
* gamma_k's radius runs exactly from 0.2 to 1.2 (eq. urchin-warping); the adaptive mesh resolves every
  element to the tolerance, refines more for a tighter tolerance, and its area converges.
"""
import math

import numpy as np
import pytest

from synth import (adaptive_flat_mesh, bisect_flat, conical_rule, flat_mesh, map_tail, surface_from_flat,
                   urchin_radius)
from synth.surfaces import _GEO_IJ, _orthonormal_by_degree, _tail_of_geometry


def _exact(a, b):
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


@pytest.mark.parametrize("n", [3, 5])
def test_conical_rule_degree(n):
    u, v, w = conical_rule(n)
    for a in range(2 * n):
        for b in range(2 * n - a):
            assert abs(np.sum(w * u ** a * v ** b) - _exact(a, b)) < 1e-15
    worst = max(abs(np.sum(w * u ** a * v ** (2 * n - a)) - _exact(a, 2 * n - a)) for a in range(2 * n + 1))
    assert worst > 1e-8


def test_basis_is_orthonormal_and_hierarchical():
    u, v, w, B, deg = _orthonormal_by_degree()
    assert np.abs((B * w) @ B.T - np.eye(15)).max() < 1e-13
    assert list(deg) == sorted(deg) and list(np.bincount(deg)) == [1, 2, 3, 4, 5]
    # the functions of degree <= d span the polynomials of degree <= d: a monomial of degree d is
    # reproduced by them exactly
    for d in range(5):
        for a in range(d + 1):
            f = u ** a * v ** (d - a)
            keep = B[deg <= d]
            proj = (keep * w) @ f
            assert np.abs(proj @ keep - f).max() < 1e-12


def _nodes():
    return np.array([(i / 4.0, j / 4.0) for i, j in _GEO_IJ])


def test_tail_of_polynomial_maps():
    p = _nodes()
    u, v = p[:, 0], p[:, 1]
    rng = np.random.default_rng(0)
    quad = np.stack([rng.normal() + rng.normal() * u + rng.normal() * v + rng.normal() * u * v + rng.normal() * u * u
                     + rng.normal() * v * v for _ in range(3)], -1)
    assert _tail_of_geometry(quad[None])[0] < 1e-14
    cub = np.stack([u ** 3, v ** 3, u * u * v], -1)
    t1 = _tail_of_geometry((quad + 1e-3 * cub)[None])[0]
    t2 = _tail_of_geometry((quad + 2e-3 * cub)[None])[0]
    assert 1e-7 < t1 < 1e-3 and abs(t2 / t1 - 2.0) < 1e-2  # the cubic part alone, linear in its size


def test_tail_decays_cubically_on_the_sphere():
    f = flat_mesh(2)
    tails = [map_tail(f).max()]
    for _ in range(2):
        f = bisect_flat(f, np.ones(len(f), bool))
        tails.append(map_tail(f).max())
    assert tails[0] / tails[1] > 6.0 and tails[1] / tails[2] > 6.0


@pytest.mark.parametrize("k", [2, 5, 8])
def test_urchin_radius_range(k):
    r = urchin_radius(k)
    rng = np.random.default_rng(k)
    x = rng.normal(size=(3, 200000))
    x /= np.linalg.norm(x, axis=0)
    vals = r(x)
    assert vals.min() >= 0.2 - 1e-12 and vals.max() <= 1.2 + 1e-12
    assert vals.min() < 0.2 + 2e-3 and vals.max() > 1.2 - 2e-3


def test_adaptive_mesh_of_an_urchin():
    r = urchin_radius(4)
    f3, h3 = adaptive_flat_mesh(r, 1e-3)
    f4, h4 = adaptive_flat_mesh(r, 1e-4)
    assert map_tail(f3, r).max() <= 1e-3 and map_tail(f4, r).max() <= 1e-4
    assert len(f4) > 2 * len(f3) and h3[-1] == 0 and h4[-1] == 0
    # element sizes vary: the mesh is adaptive, not uniform
    area = 0.5 * np.linalg.norm(np.cross(f4[:, 1] - f4[:, 0], f4[:, 2] - f4[:, 0]), axis=1)
    assert area.max() / area.min() >= 4.0 - 1e-9
    a3 = surface_from_flat(f3, r).src_w.sum()
    a4 = surface_from_flat(f4, r).src_w.sum()
    a5 = surface_from_flat(adaptive_flat_mesh(r, 1e-5)[0], r).src_w.sum()
    assert abs(a4 - a5) < abs(a3 - a5) and abs(a4 - a5) / a5 < 1e-5
