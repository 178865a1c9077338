"""Pins of the oracle's target association (Section 3.4, Algorithm 3, with the area queries of
Appendix A, Algorithm 5) against the definition evaluated over all pairs, without a tree (no GPU).

A target is endangered when some source s lies within its danger radius eta/2; an endangered target
goes to the closest center c with |t - c| <= r_c (1 + eps) on its preferred side (the side of
(t - s*) . n(s*) for the nearest source s*), ties to the lower center index; endangered targets without
such a center are flagged.  If the oracle's area queries missed a leaf, a target would lose a source
or a center and the comparison would fail.
"""
import numpy as np
import pytest

import oracle as O
from synth import danger_radius, make_surface, near_surface_points, star_radius, volume_points
from synth.surfaces import STAR_Y63

EPS = 0.05


def _brute(s, t, eps, sides=True):
    rd = danger_radius(s)
    nt = t.shape[1]
    tc = np.full(nt, -1, np.int32)
    fl = np.zeros(nt, bool)
    for i in range(nt):
        x = t[:, i]
        ds = np.sqrt(((s.src_xyz - x[:, None]) ** 2).sum(axis=0))
        if not np.any(ds <= rd):
            continue
        j = int(np.argmin(ds))  # first index among equals
        side = 1 if np.dot(x - s.src_xyz[:, j], s.src_n[:, j]) > 0 else -1
        dc = np.sqrt(((s.ctr_xyz - x[:, None]) ** 2).sum(axis=0))
        ok = dc <= s.ctr_r * (1.0 + eps)
        if sides:
            ok &= s.ctr_side == side
        if ok.any():
            cand = np.nonzero(ok)[0]
            tc[i] = cand[np.argmin(dc[cand])]
        else:
            fl[i] = True
    return tc, fl


@pytest.mark.parametrize("n_max,sides", [(8, True), (32, True), (16, False)])
def test_association_matches_the_definition(n_max, sides):
    s = make_surface(3, star_radius(STAR_Y63))
    t = np.concatenate([near_surface_points(s, 1500, seed=4), volume_points(300, seed=5, box=1.6)], axis=1)
    T = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, t, n_max=n_max, t_f=0.9)
    tc, fl = O.assoc_targets(T, s.src_xyz, danger_radius(s), s.src_n if sides else None, s.ctr_xyz, s.ctr_r,
                             s.ctr_side if sides else None, t, EPS)
    tb, fb = _brute(s, t, EPS, sides)
    assert np.array_equal(tc, tb)
    assert np.array_equal(fl, fb)
    # a non-trivial case: many associated targets on both sides, some flagged, many not endangered
    assoc = tc >= 0
    assert assoc.sum() > 500 and (tc < 0).sum() > 100
    if sides:
        assert len(set(s.ctr_side[tc[assoc]])) == 2


def test_larger_tolerance_associates_more():
    s = make_surface(3, star_radius(STAR_Y63))
    t = near_surface_points(s, 1500, seed=6)
    T = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, t, n_max=16, t_f=0.9)
    args = (T, s.src_xyz, danger_radius(s), s.src_n, s.ctr_xyz, s.ctr_r, s.ctr_side, t)
    tc0, fl0 = O.assoc_targets(*args, 0.0)
    tc1, fl1 = O.assoc_targets(*args, 0.5)
    assert fl1.sum() < fl0.sum()
    assert np.all((tc0 >= 0) <= (tc1 >= 0))  # associated at eps = 0 stays associated
