"""Pins of the oracle's octree (Algorithm 4 Stage 1) and interaction lists (Section 5.2),
checked against the definitions themselves, written independently here in numpy (no GPU).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
TF = GOLD["tf_experiments"]["value"]


def _tree(surf, n_max=32, tf=TF):
    return O.build_tree(surf.src_xyz, surf.ctr_xyz, surf.ctr_r, surf.tgt_xyz, n_max=n_max, t_f=tf)


def _morton(level, c):
    key = 0
    for bit in range(level - 1, -1, -1):
        for d in (2, 1, 0):
            key = (key << 1) | ((int(c[d]) >> bit) & 1)
    return key


def _fits(x, r, cen, h, tf):
    return math.sqrt(sum((x[d] - cen[d]) ** 2 for d in range(3))) + r <= math.sqrt(3.0) * h * (1.0 + tf)


@pytest.mark.parametrize("n_max", [8, 32, 64])
def test_tree_invariants(star_small, n_max):
    s = star_small
    T = _tree(s, n_max)
    nb = T.n_boxes
    R, c0 = T.root_radius, T.root_center
    # root contains every particle and every expansion ball
    assert np.all(np.abs(s.src_xyz - c0[:, None]) <= R)
    assert np.all(np.abs(s.ctr_xyz - c0[:, None]).max(axis=0) + s.ctr_r <= R)
    # canonical (level, Morton) order, exact dyadic geometry, children in octant order
    keys = [(T.level[b], _morton(T.level[b], T.coords[b])) for b in range(nb)]
    assert keys == sorted(keys)
    for b in range(nb):
        lev = T.level[b]
        h = R / 2 ** lev
        assert T.radius[b] == h
        assert np.all(T.center[b] == c0 - R + (2 * T.coords[b] + 1) * h)
        for o in range(8):
            ch = T.child[b, o]
            if ch >= 0:
                assert T.parent[ch] == b and T.level[ch] == lev + 1
                assert np.all(T.coords[ch] == 2 * T.coords[b] + np.array([o & 1, (o >> 1) & 1, (o >> 2) & 1]))
    leaf = np.all(T.child < 0, axis=1)
    # points live in leaves, inside their box
    for xyz, own in ((s.src_xyz, T.src_owner), (s.tgt_xyz, T.tgt_owner)):
        assert np.all(leaf[own])
        lo, hi = T.center[own] - T.radius[own, None], T.center[own] + T.radius[own, None]
        assert np.all((xyz.T >= lo) & (xyz.T <= hi))
    # each center sits in the deepest box whose TCR holds its ball
    for i in range(s.n_ctr):
        b = T.ctr_owner[i]
        x, r = s.ctr_xyz[:, i], s.ctr_r[i]
        if b != 0:
            assert _fits(x, r, T.center[b], T.radius[b], TF)
        if not leaf[b]:
            o = sum(1 << d for d in range(3) if x[d] >= T.center[b, d])
            hc = T.radius[b] / 2
            cc = T.center[b] + np.where([(o >> d) & 1 for d in range(3)], hc, -hc)
            assert not _fits(x, r, cc, hc, TF)
    # leaves own at most n_max particles unless nothing could move
    owned = np.bincount(T.src_owner, minlength=nb) + np.bincount(T.tgt_owner, minlength=nb) + \
        np.bincount(T.ctr_owner, minlength=nb)
    for b in np.nonzero(leaf & (owned > n_max))[0]:
        assert np.bincount(T.src_owner, minlength=nb)[b] == 0 and np.bincount(T.tgt_owner, minlength=nb)[b] == 0
    # non-leaf boxes own centers only
    assert np.all(leaf[T.src_owner]) and np.all(leaf[T.tgt_owner])
    assert T.n_overfull == 0


def _ancestors(T, b):
    out = []
    w = T.parent[b]
    while w >= 0:
        out.append(w)
        w = T.parent[w]
    return out


@pytest.mark.parametrize("surf_name,n_max", [("sphere80", 16), ("sphere80", 32), ("star_small", 32)])
def test_fast_lists_equal_literal_definitions(surf_name, n_max, request):
    s = request.getfixturevalue(surf_name)
    T = _tree(s, n_max)
    fast, slow = O.build_lists(T), O.build_lists(T, slow=True)
    for k in O.LIST_NAMES:
        assert np.array_equal(fast.start[k], slow.start[k]), k
        assert np.array_equal(fast.idx[k], slow.idx[k]), k


def test_list_size_lemmas(star_small):
    T = _tree(star_small, 16)
    L = O.build_lists(T)
    sizes = {k: np.diff(L.start[k]) for k in O.LIST_NAMES}
    assert sizes["V"].max() <= GOLD["list2_max"]["value"]
    assert sizes["Xclose"].max() <= GOLD["list4_close_max"]["value"]
    assert sizes["Xfar"].max() <= GOLD["list4_far_max"]["value"]


@pytest.mark.parametrize("surf_name,n_max", [("sphere80", 16), ("star_small", 32)])
def test_partition_of_sources(surf_name, n_max, request):
    """Every source leaf reaches every target box exactly once: directly (U, W-close,
    X-close), through a List 3 far multipole, or through the local expansion of the box
    or an ancestor (List 2 and List 4 far)."""
    s = request.getfixturevalue(surf_name)
    T = _tree(s, n_max)
    L = O.build_lists(T)
    nb = T.n_boxes
    leaf = np.all(T.child < 0, axis=1)
    has_src = np.bincount(T.src_owner, minlength=nb) > 0
    src_leaves = np.nonzero(leaf & has_src)[0]
    # leaves below each box (including itself)
    below = [set() for _ in range(nb)]
    for b in src_leaves:
        w = b
        while w >= 0:
            below[w].add(b)
            w = T.parent[w]
    targets = set(T.ctr_owner.tolist()) | set(T.tgt_owner.tolist())
    for b in targets:
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
        assert set(cnt.values()) == {1}, (b, {k: v for k, v in cnt.items() if v != 1})


def test_adequate_separation_of_far_lists(star_small):
    """W-far boxes d satisfy d < TCR(b) in l2; X-far boxes d satisfy TCR(b) < d in l-inf."""
    T = _tree(star_small, 16)
    L = O.build_lists(T)
    for b in range(T.n_boxes):
        tcr = math.sqrt(3.0) * T.radius[b] * (1 + TF)
        for d in L.of("Wfar", b):
            assert np.linalg.norm(T.center[d] - T.center[b]) - tcr >= 3 * T.radius[d]
        for d in L.of("Wclose", b):
            assert np.linalg.norm(T.center[d] - T.center[b]) - tcr < 3 * T.radius[d]
        for d in L.of("Xfar", b):
            assert np.abs(T.center[b] - T.center[d]).max() - T.radius[d] >= 3 * T.radius[b] * (1 + TF)
        for d in L.of("Xclose", b):
            assert np.abs(T.center[b] - T.center[d]).max() - T.radius[d] < 3 * T.radius[b] * (1 + TF)
