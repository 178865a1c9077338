"""Pins of the oracle's tree variants (no GPU), checked against their definitions written
independently here in numpy:

* the l-infinity target confinement region of the two-dimensional method, which Table
  l2-comparison sets against the l2 TCR of Section 5.2.2: a center is owned by the deepest box
  whose cube of radius |b|(1+t_f) holds its ball, and List 3 far boxes d satisfy
  d < TCR(b) in the l-infinity distance;
* level restriction (Remark "Effect of level-restriction on List 3 complexity", Section 5.3):
  adjacent leaves differ by at most one level, the restricted tree refines the plain one, and
  every box the restriction split has a box two or more levels finer beside it.

The lists of every variant equal their literal definitions and still route every source leaf to
every target box exactly once, and Algorithm 4 on a variant tree still converges to direct QBX.
"""
import math

import numpy as np
import pytest

import oracle as O
from synth import real_ylm

from conftest import rel_linf

TF = 0.9
VARIANTS = [(True, False), (False, True), (True, True)]


def _tree(s, n_max, linf, restrict, tf=TF):
    return O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, s.tgt_xyz, n_max=n_max, t_f=tf, linf_tcr=linf,
                        level_restrict=restrict)


def _fits(x, r, cen, h, tf, linf):
    if linf:
        return float(np.max(np.abs(x - cen))) + r <= h * (1.0 + tf)
    return math.sqrt(float(np.sum((x - cen) ** 2))) + r <= math.sqrt(3.0) * h * (1.0 + tf)


def _extent(T, b, lf):
    sh = lf - T.level[b]
    return T.coords[b] << sh, (T.coords[b] + 1) << sh


def _touching(T, a, b, lf):
    """Closed cubes meet and interiors are disjoint (exact integer test)."""
    la, ha = _extent(T, a, lf)
    lb, hb = _extent(T, b, lf)
    closed = np.all(la <= hb) and np.all(lb <= ha)
    open_ = np.all(la < hb) and np.all(lb < ha)
    return bool(closed and not open_)


def _stuck(T, s, b, tf, linf):
    """No particle of b could move to a child: b owns only centers, none fits its octant child's TCR."""
    if np.any(T.src_owner == b) or np.any(T.tgt_owner == b):
        return False
    hc = T.radius[b] / 2
    for i in np.nonzero(T.ctr_owner == b)[0]:
        x = s.ctr_xyz[:, i]
        o = [1 if x[d] >= T.center[b, d] else 0 for d in range(3)]
        cc = T.center[b] + np.where(o, hc, -hc)
        if _fits(x, s.ctr_r[i], cc, hc, tf, linf):
            return False
    return True


@pytest.mark.parametrize("linf,restrict", VARIANTS)
@pytest.mark.parametrize("n_max", [8, 32])
def test_variant_tree_invariants(star_small, n_max, linf, restrict):
    s = star_small
    T = _tree(s, n_max, linf, restrict)
    nb = T.n_boxes
    R, c0 = T.root_radius, T.root_center
    keys = [(int(T.level[b]), tuple(T.coords[b])) for b in range(nb)]
    assert len(set(keys)) == nb
    # (level, Morton) order: same-level boxes in Morton order, levels ascending
    def morton(lev, c):
        k = 0
        for bit in range(lev - 1, -1, -1):
            for d in (2, 1, 0):
                k = (k << 1) | ((int(c[d]) >> bit) & 1)
        return k
    order = [(int(T.level[b]), morton(int(T.level[b]), T.coords[b])) for b in range(nb)]
    assert order == sorted(order)
    for b in range(nb):
        h = R / 2 ** T.level[b]
        assert T.radius[b] == h
        assert np.all(T.center[b] == c0 - R + (2 * T.coords[b] + 1) * h)
        for o in range(8):
            ch = T.child[b, o]
            if ch >= 0:
                assert T.parent[ch] == b and T.level[ch] == T.level[b] + 1
    leaf = np.all(T.child < 0, axis=1)
    # points in leaves, inside their box
    for xyz, own in ((s.src_xyz, T.src_owner), (s.tgt_xyz, T.tgt_owner)):
        assert np.all(leaf[own])
        lo, hi = T.center[own] - T.radius[own, None], T.center[own] + T.radius[own, None]
        assert np.all((xyz.T >= lo) & (xyz.T <= hi))
    # each center in the deepest box whose TCR (of this variant's shape) holds its ball
    for i in range(s.n_ctr):
        b = T.ctr_owner[i]
        x, r = s.ctr_xyz[:, i], s.ctr_r[i]
        if b != 0:
            assert _fits(x, r, T.center[b], T.radius[b], TF, linf)
        if not leaf[b]:
            o = [1 if x[d] >= T.center[b, d] else 0 for d in range(3)]
            hc = T.radius[b] / 2
            assert not _fits(x, r, T.center[b] + np.where(o, hc, -hc), hc, TF, linf)
    if restrict:
        lf = int(T.level.max())
        leaves = np.nonzero(leaf)[0]
        sh = (lf - T.level[leaves])[:, None]
        lo, hi = T.coords[leaves] << sh, (T.coords[leaves] + 1) << sh
        for j, b in enumerate(leaves):
            closed = np.all((lo <= hi[j]) & (lo[j] <= hi), axis=1)
            deep = T.level[leaves] >= T.level[b] + 2
            for a in leaves[closed & deep]:  # leaves never nest: closed contact means adjacent
                assert _touching(T, a, b, lf) and _stuck(T, s, b, TF, linf), (b, a)


def test_linf_tcr_is_a_different_tree(star_small):
    """The cube of radius |b|(1+t_f) lies inside the ball of radius sqrt(3)|b|(1+t_f), so with
    the l-infinity TCR fewer centers descend: every center sits at its l2 depth or above."""
    s = star_small
    T2 = _tree(s, 16, False, False)
    Ti = _tree(s, 16, True, False)
    assert Ti.n_boxes != T2.n_boxes
    assert np.all(Ti.level[Ti.ctr_owner] <= T2.level[T2.ctr_owner])
    assert np.any(Ti.level[Ti.ctr_owner] < T2.level[T2.ctr_owner])


@pytest.mark.parametrize("linf", [False, True])
def test_level_restriction_refines_and_is_needed(star_small, linf):
    s = star_small
    T0 = _tree(s, 8, linf, False)
    T1 = _tree(s, 8, linf, True)
    k0 = {(int(T0.level[b]), tuple(T0.coords[b])): b for b in range(T0.n_boxes)}
    k1 = {(int(T1.level[b]), tuple(T1.coords[b])): b for b in range(T1.n_boxes)}
    assert set(k0) <= set(k1)
    assert T1.n_boxes > T0.n_boxes  # this surface needs restriction at n_max = 8
    leaf0 = np.all(T0.child < 0, axis=1)
    leaf1 = np.all(T1.child < 0, axis=1)
    lf = int(T1.level.max())
    split_by_restriction = []
    for key, b in k1.items():
        if key not in k0:
            # new boxes lie below a leaf of the plain tree
            w = T1.parent[b]
            while (int(T1.level[w]), tuple(T1.coords[w])) not in k0:
                w = T1.parent[w]
            assert leaf0[k0[(int(T1.level[w]), tuple(T1.coords[w]))]]
        was_leaf = key not in k0 or leaf0[k0[key]]
        if was_leaf and not leaf1[b]:
            split_by_restriction.append(b)
    assert split_by_restriction
    # every such split had a box two or more levels finer touching it
    for b in split_by_restriction:
        assert any(T1.level[a] >= T1.level[b] + 2 and _touching(T1, a, b, lf) for a in range(T1.n_boxes)), b


def test_level_restriction_of_a_uniform_tree_changes_nothing():
    """Sources on a regular lattice give a tree whose leaves are all on one level: nothing to do."""
    g = (np.arange(8) + 0.5) / 8.0
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    src = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    ctr = np.zeros((3, 0))
    T0 = O.build_tree(src, ctr, np.zeros(0), np.zeros((3, 0)), n_max=1)
    T1 = O.build_tree(src, ctr, np.zeros(0), np.zeros((3, 0)), n_max=1, level_restrict=True)
    assert T0.n_boxes == T1.n_boxes
    for k in ("level", "coords", "parent", "child", "src_owner"):
        assert np.array_equal(getattr(T0, k), getattr(T1, k))


@pytest.mark.parametrize("linf,restrict", VARIANTS)
def test_variant_fast_lists_equal_literal_definitions(sphere80, linf, restrict):
    T = _tree(sphere80, 8, linf, restrict)
    fast, slow = O.build_lists(T), O.build_lists(T, slow=True)
    for k in O.LIST_NAMES:
        assert np.array_equal(fast.start[k], slow.start[k]), k
        assert np.array_equal(fast.idx[k], slow.idx[k]), k


def _ancestors(T, b):
    out = []
    w = T.parent[b]
    while w >= 0:
        out.append(w)
        w = T.parent[w]
    return out


@pytest.mark.parametrize("linf,restrict", VARIANTS)
def test_variant_partition_of_sources(sphere80, linf, restrict):
    """Every source leaf reaches every target box exactly once (direct lists, List 3 far
    multipoles, or local expansions of the box or an ancestor)."""
    s = sphere80
    T = _tree(s, 16, linf, restrict)
    L = O.build_lists(T)
    nb = T.n_boxes
    leaf = np.all(T.child < 0, axis=1)
    src_leaves = np.nonzero(leaf & (np.bincount(T.src_owner, minlength=nb) > 0))[0]
    below = [set() for _ in range(nb)]
    for b in src_leaves:
        w = b
        while w >= 0:
            below[w].add(b)
            w = T.parent[w]
    for b in set(T.ctr_owner.tolist()) | set(T.tgt_owner.tolist()):
        cnt = dict.fromkeys(src_leaves.tolist(), 0)
        for name in ("U", "Wclose", "Xclose"):
            for d in L.of(name, b):
                cnt[d] += 1
        for d in L.of("Wfar", b):
            for lf in below[d]:
                cnt[lf] += 1
        for w in [b] + _ancestors(T, b):
            for d in L.of("V", w):
                for lf in below[d]:
                    cnt[lf] += 1
            for d in L.of("Xfar", w):
                cnt[d] += 1
        assert set(cnt.values()) == {1}, b


def test_linf_far_list_separation(star_small):
    """With the l-infinity TCR, List 3 far boxes d satisfy: l-infinity distance from c_d to the
    boundary of the cube of radius |b|(1+t_f) is >= 3|d|; List 3 close leaves do not."""
    T = _tree(star_small, 16, True, False)
    L = O.build_lists(T)
    n_far = 0
    for b in range(T.n_boxes):
        tcr = T.radius[b] * (1 + TF)
        for d in L.of("Wfar", b):
            assert np.abs(T.center[d] - T.center[b]).max() - tcr >= 3 * T.radius[d]
            n_far += 1
        for d in L.of("Wclose", b):
            assert np.abs(T.center[d] - T.center[b]).max() - tcr < 3 * T.radius[d]
    assert n_far > 0


def test_variant_fmm_converges_to_direct_qbx(sphere80):
    s = sphere80
    sig = real_ylm(2, 1, s.src_xyz)
    ref = O.direct_eval(s.src_xyz, s.src_w, sig, None, s.src_n, s.ctr_xyz, s.tgt_xyz, s.tgt_ctr, 5)
    T = _tree(s, 32, True, True)
    L = O.build_lists(T)
    errs = {p: rel_linf(O.fmm_eval(T, L, s.src_xyz, s.src_w, sig, None, s.src_n, s.ctr_xyz, s.tgt_xyz, s.tgt_ctr,
                                   5, p), ref) for p in (3, 6, 9)}
    assert errs[3] > errs[6] > errs[9]
    assert errs[9] <= errs[3] * 0.7711 ** 6
