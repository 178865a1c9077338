"""Input generator checks (no GPU): quadrature exactness, geometry, seeded point sets."""
import math

import numpy as np

from synth import danger_radius, make_surface, near_surface_points, triangle_rule, volume_points
from synth.surfaces import STAR_Y63, star_radius


def test_triangle_rule_monomial_exactness():
    u, v, w = triangle_rule()
    assert u.size == 15
    for a in range(6):
        for b in range(6 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.sum(w * u ** a * v ** b) - exact) < 1e-15


def test_sphere_area_normals_and_radii(sphere320):
    s = sphere320
    assert s.n_src == 4800 and s.n_ctr == 9600
    assert abs(s.src_w.sum() - 4 * math.pi) < 1e-5
    assert np.allclose(np.linalg.norm(s.src_n, axis=0), 1.0)
    assert np.all(np.sum(s.src_n * s.src_xyz, axis=0) > 0.99)
    # radius = half the element size: flat sub-triangles of the icosahedron have edges ~ 0.27
    assert 0.1 < s.ctr_r.min() and s.ctr_r.max() < 0.2
    d = np.linalg.norm(s.ctr_xyz - np.concatenate([s.src_xyz, s.src_xyz], axis=1), axis=0)
    assert np.allclose(d, s.ctr_r)


def test_point_sets_are_seeded_and_placed():
    s = make_surface(4, star_radius(STAR_Y63))
    v = volume_points(500, seed=2)
    assert v.shape == (3, 500) and np.array_equal(v, volume_points(500, seed=2))
    assert np.all(np.abs(v) <= 2.0)
    p = near_surface_points(s, 400, seed=3)
    assert np.array_equal(p, near_surface_points(s, 400, seed=3))
    rd = danger_radius(s)
    assert np.allclose(rd, 0.5 * s.elem_eta[s.src_elem]) and np.all(rd > 0)
    # every point lies within a few danger radii of some source
    d = np.min(np.linalg.norm(p[:, :, None] - s.src_xyz[:, None, :], axis=0), axis=1)
    assert np.all(d <= 4.0 * rd.max())


def test_batched_specs_follow_the_recipe():
    from synth import batched_specs

    a = batched_specs(64, seed=5)
    assert a == batched_specs(64, seed=5)  # seeded
    assert len(a) == 64
    for n, terms, dseed in a:
        assert 4 <= n <= 26  # 300 n^2 sources: 4,800 .. 202,800
        (amp, k, m), = terms
        assert 2 <= k <= 10 and m == k // 2 and 0.1 <= amp <= 0.4
    assert [d for _, _, d in a] == list(range(500, 564))
    total = sum(300 * n * n for n, _, _ in a)
    assert 1_000_000 < total < 6_000_000


def test_upsampled_source_quadrature():
    """f^2 copies of the rule on the sub-triangles: same area, same centers, finer sources."""
    s1 = make_surface(2)
    s3 = make_surface(2, upsample=3)
    assert s3.n_src == 9 * s1.n_src and s3.n_ctr == s1.n_ctr
    assert np.array_equal(s3.ctr_xyz, s1.ctr_xyz) and np.array_equal(s3.tgt_xyz, s1.tgt_xyz)
    assert abs(s3.src_w.sum() - s1.src_w.sum()) < 1e-4 * s1.src_w.sum()
    assert np.allclose(np.linalg.norm(s3.src_n, axis=0), 1.0)
    assert np.allclose(np.linalg.norm(s3.src_xyz, axis=0), 1.0, atol=2e-3)  # on the (interpolated) sphere
