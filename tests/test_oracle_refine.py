"""Pins of the oracle's refinement tests (Algorithms 1 and 2, Sections 3.2-3.3) and of the
geometry they read (no GPU).

* Threshold semantics: Algorithm 1 marks a source strictly inside (1 - eps) r, Algorithm 2 a
  center at most 0.5 (3/4) eta_k from a source.
* A convex surface at uniform resolution needs no refinement: a center x +- r n of the unit
  sphere is at distance >= r from every point of the sphere, so no source lies inside
  (1 - eps) r, and no center lies within 0.375 eta of a source when eta varies by less than 4/3.
* Two spheres a gap g < r apart: an element of the first sphere is marked by Algorithm 1 exactly
  where its centers come closer to the second sphere than (1 - eps) r, up to the sampling of that
  sphere by source nodes (closed-form distance |c - c_B| - 1).
* After one element of the sphere is bisected, Algorithm 2 marks elements around it (the paper's
  'buffer zone'), never the children themselves.
* Geometry: the principal curvatures of the degree-4 element maps converge to 1/R on a sphere of
  radius R, so the scaled curvature max(|k1|, |k2|) eta tends to eta / R.
"""
import numpy as np
import pytest

import oracle as O
from synth import bisect_flat, flat_mesh, make_surface, scaled_curvature, surface_from_flat

EPS = 0.025


def test_threshold_semantics():
    r = 1.0
    edge = (1.0 - EPS) * r
    c = np.zeros((3, 1))
    for x, want in ((edge, False), (np.nextafter(edge, 0.0), True), (0.5, True), (2.0, False)):
        s = np.array([[x], [0.0], [0.0]])
        got = O.refine_marks(0, s, c, np.array([r]), np.array([0]), 1, eps=EPS)
        assert bool(got[0]) == want, x
    s = np.zeros((3, 1))
    for x, want in ((0.375, True), (np.nextafter(0.375, 1.0), False), (0.1, True)):
        cc = np.array([[x], [0.0], [0.0]])
        got = O.refine_marks(1, s, cc, np.array([9.0]), np.array([0]), 1, elem_eta=np.array([1.0]))
        assert bool(got[0]) == want, x


@pytest.mark.parametrize("n_sub", [2, 3, 5])
def test_uniform_sphere_needs_no_refinement(n_sub):
    s = make_surface(n_sub)
    assert s.elem_eta.max() / s.elem_eta.min() < 4.0 / 3.0
    assert not O.refine_marks(0, s.src_xyz, s.ctr_xyz, s.ctr_r, s.ctr_elem, s.n_elem, eps=EPS).any()
    assert not O.refine_marks(1, s.src_xyz, s.ctr_xyz, s.ctr_r, s.src_elem, s.n_elem, s.elem_eta).any()


def _two_spheres(n_sub, gap):
    f = flat_mesh(n_sub)
    a = surface_from_flat(f)
    b = surface_from_flat(f, offset=(2.0 + gap, 0.0, 0.0))
    src = np.concatenate([a.src_xyz, b.src_xyz], 1)
    ctr = np.concatenate([a.ctr_xyz, b.ctr_xyz], 1)
    cr = np.concatenate([a.ctr_r, b.ctr_r])
    ce = np.concatenate([a.ctr_elem, b.ctr_elem + a.n_elem])
    return a, b, src, ctr, cr, ce


@pytest.mark.parametrize("gap", [0.02, 0.08])
def test_two_spheres_interfering_sources(gap):
    a, b, src, ctr, cr, ce = _two_spheres(4, gap)
    K = a.n_elem
    marks = O.refine_marks(0, src, ctr, cr, ce, 2 * K, eps=EPS)
    cB = np.array([2.0 + gap, 0.0, 0.0])
    # how far the second sphere's nodes stray from the exact sphere, and how coarsely they sample it:
    # every point of an element map lies within rho_e of one of the element's 15 nodes (measured on
    # 240 points per element), plus the spacing of those points and the deviation from the sphere
    fine = surface_from_flat(flat_mesh(4), offset=(2.0 + gap, 0.0, 0.0), upsample=4)
    pts = fine.src_xyz.T.reshape(K, -1, 3)
    nodes = b.src_xyz.T.reshape(K, 15, 3)
    rho_e = np.linalg.norm(pts[:, :, None, :] - nodes[:, None, :, :], axis=-1).min(axis=2).max()
    dev = max(np.abs(np.linalg.norm(b.src_xyz.T - cB, axis=1) - 1.0).max(),
              np.abs(np.linalg.norm(fine.src_xyz.T - cB, axis=1) - 1.0).max())
    rho = rho_e + b.elem_eta.max() / 8.0 + dev
    dist = np.abs(np.linalg.norm(a.ctr_xyz.T - cB, axis=1) - 1.0)  # centers of the first sphere to the second
    lim = (1.0 - EPS) * a.ctr_r
    sure = np.zeros(K, bool)
    never = np.ones(K, bool)
    np.logical_or.at(sure, a.ctr_elem, dist + rho < lim)
    np.logical_and.at(never, a.ctr_elem, dist - dev >= lim)
    assert sure.any() and never.any()
    assert np.all(marks[:K][sure]) and not np.any(marks[:K][never])
    # by symmetry the second sphere's elements facing the first are marked the same way
    assert marks[:K].sum() == marks[K:].sum()


def test_quadrature_resolution_buffer_zone():
    f = flat_mesh(3)
    bis = np.zeros(len(f), bool)
    bis[7] = True
    f2 = bisect_flat(f, bis)
    s = surface_from_flat(f2)
    marks = O.refine_marks(1, s.src_xyz, s.ctr_xyz, s.ctr_r, s.src_elem, s.n_elem, s.elem_eta)
    kids = np.arange(len(f) - 1, len(f2))
    assert not marks[kids].any()
    assert 0 < marks.sum() <= 12  # at most the elements that share a vertex with the bisected one
    # marked elements touch the bisected one (share a vertex of its flat triangle)
    parent = f[7]
    for k in np.nonzero(marks)[0]:
        d = np.linalg.norm(f2[k][:, None, :] - parent[None, :, :], axis=-1)
        assert d.min() < 1e-12, k


def test_bisection_halves_eta():
    f = flat_mesh(3)
    bis = np.zeros(len(f), bool)
    bis[[0, 5]] = True
    s1 = surface_from_flat(f)
    s2 = surface_from_flat(bisect_flat(f, bis))
    kids = s2.elem_eta[-8:].reshape(2, 4)
    np.testing.assert_allclose(kids / s1.elem_eta[[0, 5]][:, None], 0.5, rtol=0.1)  # curved maps: about half
    np.testing.assert_array_equal(s2.elem_eta[:len(f) - 2], s1.elem_eta[~bis])


@pytest.mark.parametrize("R", [1.0, 2.5])
def test_scaled_curvature_on_spheres(R):
    k2 = scaled_curvature(flat_mesh(4), scale=R)
    k8 = scaled_curvature(flat_mesh(8), scale=R)
    e2 = make_surface(4, scale=R).elem_eta
    e8 = make_surface(8, scale=R).elem_eta
    err2 = np.abs(k2 / e2 - 1.0 / R).max() * R
    err8 = np.abs(k8 / e8 - 1.0 / R).max() * R
    assert err8 < 0.01 and err8 < err2 / 4  # converges to 1/R, degree-4 maps: at least second order
