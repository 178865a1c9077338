"""Pins of the oracle's cost model and of its learned-order functions (no GPU).

* Interaction counts and modeled operation counts (Table ilist-operation-counts and Table
  complexity-analysis) on two small trees whose boxes and lists are worked out by hand below
  from the definitions of Section 5.2 (the hand analysis is written next to each expected number).
* The order network's gradient against central differences of the oracle's own FP64 loss, for
  every parameter block.
* Sweep labels and the prediction-to-order map against hand-made cases that follow from their
  definitions (the network and its orders are not in the paper).
"""
import numpy as np
import pytest

import oracle as O

TF = 0.9

# The trees below live in the root box [-1, 1]^3: anchors at (+-0.75, +-0.75, +-0.75) make the bounding
# box [-0.75, 0.75]^3 (midpoint 0, largest half extent 0.75, so R = 1 because 1.25 x 0.75 <= 1 < 2 x 0.9375).
# A level-l box has half width 2^-l and integer coordinates i with [-1 + i 2^(1-l), -1 + (i+1) 2^(1-l)].
# n_max = 1: a box owning two or more particles splits.


def _anchors(octants):
    pts = []
    for o in octants:
        pts.append([0.75 if (o >> d) & 1 else -0.75 for d in range(3)])
    return pts


def _build(sources, centers, radii):
    s = np.array(sources, dtype=np.float64).T.copy()
    c = np.array(centers, dtype=np.float64).T.copy()
    r = np.array(radii, dtype=np.float64)
    T = O.build_tree(s, c, r, np.zeros((3, 0)), n_max=1, t_f=TF)
    return T, O.build_lists(T)


def _box(T, level, ijk):
    for b in range(T.n_boxes):
        if T.level[b] == level and tuple(T.coords[b]) == tuple(ijk):
            return b
    raise AssertionError(f"no box {ijk} at level {level}")


def _list_boxes(T, L, name, b):
    return sorted((int(T.level[d]), tuple(int(v) for v in T.coords[d])) for d in L.of(name, b))


def _case_w():
    """Center C at (-0.7,-0.7,-0.7), r = 0.05, alone in the level-2 box (0,0,0) = [-1,-0.5]^3 (call it A).
    Sources: P1 (-0.4)^3 in level-3 box (2,2,2); P2 (-0.2)^3 and P3 (-0.1)^3 split the level-3 box (3,3,3)
    into level-4 boxes (6,6,6) and (7,7,7); S2 (0.75,-0.75,-0.75) and S3 (0.25,-0.75,-0.75) split the
    octant (+,-,-) into level-2 boxes (3,0,0) and (2,0,0); one anchor in each of the six other octants
    (level-1 leaves).  17 boxes, 11 sources, 1 center."""
    src = [[-0.4] * 3, [-0.2] * 3, [-0.1] * 3, [0.75, -0.75, -0.75], [0.25, -0.75, -0.75]]
    src += _anchors([2, 3, 4, 5, 6, 7])
    return _build(src, [[-0.7] * 3], [0.05])


def _case_x():
    """Center C at (-0.45)^3, r = 0.005, alone in the level-4 box (4,4,4) = [-0.5,-0.375]^3 (call it a).
    Sources: Pb (-0.3)^3 in level-4 box (5,5,5); Pa (-0.1)^3 in level-3 box (3,3,3); an anchor in each of
    the seven octants other than (-,-,-) (level-1 leaves).  14 boxes, 9 sources, 1 center."""
    src = [[-0.3] * 3, [-0.1] * 3] + _anchors([1, 2, 3, 4, 5, 6, 7])
    return _build(src, [[-0.45] * 3], [0.005])


def test_hand_tree_w_lists_and_counts():
    T, L = _case_w()
    assert T.n_boxes == 17 and T.n_levels == 5 and T.root_radius == 1.0 and np.all(T.root_center == 0.0)
    A = int(T.ctr_owner[0])
    assert T.level[A] == 2 and tuple(T.coords[A]) == (0, 0, 0)
    # List 1: leaves adjacent to A with sources: only (2,2,2) at level 3 touches A (at the corner -0.5)
    assert _list_boxes(T, L, "U", A) == [(3, (2, 2, 2))]
    # List 2: children of the parent's 2-colleagues (all level-1 boxes) that are not 2-colleagues of A:
    # (3,0,0) is three boxes away in x; (1,1,1) and (2,0,0) are within two
    assert _list_boxes(T, L, "V", A) == [(2, (3, 0, 0))]
    # List 3: children of the 2-colleague (1,1,1) not adjacent to A: (3,3,3); it is not separated from
    # TCR(A) (sqrt(3) 0.625 - sqrt(3) 0.25 x 1.9 = 0.260 < 3 x 0.125) and not a leaf, so its children are
    # tested: (6,6,6) gives 0.152 < 0.1875 (a leaf: close), (7,7,7) gives 0.368 >= 0.1875 (far)
    assert _list_boxes(T, L, "Wclose", A) == [(4, (6, 6, 6))]
    assert _list_boxes(T, L, "Wfar", A) == [(4, (7, 7, 7))]
    # List 4: (2,0,0) (a non-adjacent 2-colleague leaf) and the six level-1 leaves (2-colleagues of the
    # parent, adjacent to it, not to A); TCR(A) is not separated from any of them
    # (max_d |c_A - c_d| - |d| = 0.75 < 3 x 0.25 x 1.9)
    assert len(L.of("Xclose", A)) == 7 and (2, (2, 0, 0)) in _list_boxes(T, L, "Xclose", A)
    assert len(L.of("Xfar", A)) == 0
    # only A owns a center (n_t = 1); every source box above holds one source
    assert O.lists_counts(T, L) == {"U": 1, "V": 1, "Wclose": 1, "Wfar": 1, "Xclose": 7, "Xfar": 0}
    q, p = 3, 5
    cost = O.lists_cost(T, L, q, p)
    want = {"U": q * q, "V": p ** 3, "Wclose": q * q, "Wfar": p ** 3, "Xclose": 7 * q * q, "Xfar": 0}
    for k, v in want.items():
        assert cost[k] == v, k
    # stage terms: N_S p^2 + N_B p^3 + 8 N_B p^3 + N_C p^3 + N_T q^2 with N_S = 11, N_B = 17, N_C = 1, N_T = 0
    assert cost["stages"] == 11 * p * p + 17 * p ** 3 + 8 * 17 * p ** 3 + p ** 3
    assert cost["total"] == sum(want.values()) + cost["stages"]


def test_hand_tree_x_lists_and_counts():
    T, L = _case_x()
    assert T.n_boxes == 14 and T.n_levels == 5
    a = int(T.ctr_owner[0])
    assert T.level[a] == 4 and tuple(T.coords[a]) == (4, 4, 4)
    b3 = _box(T, 3, (2, 2, 2))  # parent of a
    assert _list_boxes(T, L, "U", a) == [(4, (5, 5, 5))]
    assert len(L.of("V", a)) == 0 and len(L.of("Wclose", a)) == 0 and len(L.of("Wfar", a)) == 0
    # List 4 of the parent (2,2,2): the seven level-1 leaves (2-colleagues of an ancestor, adjacent to the
    # grandparent (1,1,1) at the origin, not to (2,2,2)), all close: max_d |c - c_d| - |d| = 0.375 < 0.7125
    assert len(L.of("Xclose", b3)) == 7 and len(L.of("Xfar", b3)) == 0
    # a inherits them: for a, 0.9375 - 0.5 = 0.4375 >= 3 x 0.0625 x 1.9 = 0.35625, so they are far; (3,3,3)
    # (a 2-colleague of the parent, adjacent to it, not to a) gives 0.3125 - 0.125 < 0.35625: close
    assert _list_boxes(T, L, "Xclose", a) == [(3, (3, 3, 3))]
    assert len(L.of("Xfar", a)) == 7 and all(T.level[d] == 1 for d in L.of("Xfar", a))
    # the parent owns no center, so its List 4 close entries count n_s n_t = 0; X-far counts n_s per entry
    assert O.lists_counts(T, L) == {"U": 1, "V": 0, "Wclose": 0, "Wfar": 0, "Xclose": 1, "Xfar": 7}
    q, p = 4, 6
    cost = O.lists_cost(T, L, q, p)
    assert cost["U"] == q * q and cost["Xclose"] == q * q and cost["Xfar"] == 7 * p * p
    assert cost["V"] == cost["Wclose"] == cost["Wfar"] == 0
    assert cost["stages"] == 9 * p * p + 14 * p ** 3 + 8 * 14 * p ** 3 + p ** 3


def test_counts_cover_every_source_once_per_center_box(star_small):
    """Each center's box reaches every source exactly once (Lists 1-4 of the box, Lists 2 and 4 far of
    its ancestors): so the direct pairs plus the far-routed pairs equal N_S x N_C."""
    s = star_small
    T = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, s.tgt_xyz, n_max=16, t_f=TF)
    L = O.build_lists(T)
    c = O.lists_counts(T, L)
    nb = T.n_boxes
    nsub = np.zeros(nb, np.int64)
    np.add.at(nsub, T.src_owner, 1)
    for b in range(nb - 1, 0, -1):
        nsub[T.parent[b]] += nsub[b]
    nctr = np.bincount(T.ctr_owner, minlength=nb)
    far = 0
    for b in np.nonzero(nctr)[0]:
        routed = sum(nsub[d] for d in L.of("Wfar", b))
        a = b
        while a >= 0:
            routed += sum(nsub[d] for d in L.of("V", a)) + sum(nsub[d] for d in L.of("Xfar", a))
            a = T.parent[a]
        far += nctr[b] * routed
    assert c["U"] + c["Wclose"] + c["Xclose"] + far == s.n_src * s.n_ctr


# ---------------------------------------------------------------- order network gradient


def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    P = rng.normal(size=4610) * 0.4
    x = rng.normal(size=(40, 4))
    t = rng.normal(size=(40, 2)) * 3
    g, loss = O.mlp_loss_grad_f64(P, x, t)
    # loss itself: 1/(2n) sum |y - t|^2 with y from an independent numpy forward pass
    h1 = np.tanh(x @ P[:256].reshape(64, 4).T + P[256:320])
    h2 = np.tanh(h1 @ P[320:4416].reshape(64, 64).T + P[4416:4480])
    y = h2 @ P[4480:4608].reshape(2, 64).T + P[4608:4610]
    assert loss == pytest.approx(0.5 * np.sum((y - t) ** 2) / 40, rel=1e-13)
    blocks = {"W1": (0, 256), "b1": (256, 320), "W2": (320, 4416), "b2": (4416, 4480), "W3": (4480, 4608),
              "b3": (4608, 4610)}
    h = 1e-5
    for name, (lo, hi) in blocks.items():
        idx = np.unique(np.linspace(lo, hi - 1, min(12, hi - lo)).astype(int))
        for i in idx:
            Pp, Pm = P.copy(), P.copy()
            Pp[i] += h
            Pm[i] -= h
            fd = (O.mlp_loss_grad_f64(Pp, x, t)[1] - O.mlp_loss_grad_f64(Pm, x, t)[1]) / (2 * h)
            assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (name, i, fd, g[i])
    # the float front end is the same computation on float inputs
    Pf, xf, tf_ = P.astype(np.float32), x.astype(np.float32), t.astype(np.float32)
    g32, l32 = O.mlp_loss_grad(Pf, xf, tf_)
    g64, l64 = O.mlp_loss_grad_f64(Pf.astype(np.float64), xf.astype(np.float64), tf_.astype(np.float64))
    assert np.array_equal(g32, g64) and l32 == l64


# ---------------------------------------------------------------- sweep labels


def test_order_labels_follow_their_definition():
    orders = [2, 4, 6, 8]
    cols = np.array([
        [5.0, 1.05, 1.0, 1.0],     # first column out, the rest within 0.1 of the last: 4
        [1.0, 2.0, 1.0, 1.0],      # within, out, within: the label is where it stays within: 6
        [1.0, 1.0, 1.0, 1.0],      # all equal: the lowest order, 2
        [0.0, 0.0, 0.0, 1.0],      # only the reference: 8
        [1.1, 1.1, 1.1, 1.0],      # 1.1 - 1.0 is 0.10000000000000009 > 0.1: 8
        [np.nan, 1.0, 1.0, 1.0],   # a NaN column is never within: 4
        [1.0, 1.0, np.inf, 1.0],   # an infinite column: 8
    ]).T.copy()
    assert O.order_labels(cols, orders, 0.1).tolist() == [4, 6, 2, 8, 8, 4, 8]
    # tolerance boundary is inclusive: |1.25 - 1.0| = 0.25 exactly
    v = np.array([[1.5], [1.25], [1.0]])
    assert O.order_labels(v, [3, 5, 7], 0.25).tolist() == [5]


# ---------------------------------------------------------------- prediction -> orders


def test_orders_from_predictions_follow_their_definition(star_small):
    s = star_small
    T = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, s.tgt_xyz, n_max=16, t_f=TF)
    nc, nb = s.n_ctr, T.n_boxes
    # boxes with a center somewhere below them (including their own)
    has = np.zeros(nb, bool)
    for c in range(nc):
        b = T.ctr_owner[c]
        while b >= 0 and not has[b]:
            has[b] = True
            b = T.parent[b]
    # constant predictions: ceil(3.2 + 0.5) = 4 for every center; 6.0 + 1.0 = 7 exactly -> 7 for the boxes
    pred = np.tile(np.array([3.2, 6.0], np.float32), (nc, 1))
    q, p = O.orders_from_pred(T, pred, 0.5, 1.0, 2, 12, 4, 20, 16)
    assert np.all(q == 4)
    assert np.all(p[has] == 7) and np.all(p[~has] == 16)
    # rounding up, clamping and NaN
    pred = np.array([[3.5, 2.0], [100.0, -50.0], [np.nan, np.nan], [-9.0, 30.0]], np.float32)
    pred = np.concatenate([pred, np.tile(np.array([[5.0, 4.0]], np.float32), (nc - 4, 1))])
    q, p = O.orders_from_pred(T, pred, 0.5, 0.0, 2, 12, 4, 20, 16)
    assert q[:4].tolist() == [4, 12, 12, 2]
    assert np.all(q[4:] == 6)
    # box orders: the NaN center (-> 20) dominates its box and every ancestor; center 3 (30 -> 20) too;
    # other boxes with centers get 4 (center 1: -50 -> 4; the rest: 4)
    hot = np.zeros(nb, bool)
    for c in (2, 3):
        b = T.ctr_owner[c]
        while b >= 0:
            hot[b] = True
            b = T.parent[b]
    assert np.all(p[hot] == 20) and np.all(p[has & ~hot] == 4) and np.all(p[~has] == 16)
    # point targets: their boxes and ancestors take p_hi
    tc = np.full(s.tgt_xyz.shape[1], -1, np.int32)
    tc[1:] = s.tgt_ctr[1:]
    q, p = O.orders_from_pred(T, np.tile(np.array([5.0, 5.0], np.float32), (nc, 1)), 0.0, 0.0, 2, 12, 4, 18, 16,
                              tgt_ctr=tc)
    b = T.tgt_owner[0]
    path = []
    while b >= 0:
        path.append(b)
        b = T.parent[b]
    assert np.all(p[path] == 18)
    rest = np.setdiff1d(np.nonzero(has)[0], path)
    assert np.all(p[rest] == 5)



# ---------------------------------------------------------------- network inputs


def test_center_features_on_the_unit_sphere(sphere80):
    """Unit sphere centred at the origin, one box (n_max above the particle count): the root is
    centred at 0 with |root| = R a power of two, so an interior center at distance 1 - r from the
    origin reaches (1 - r) + r = 1 from the box center (feature 2 is 1/R); an exterior one reaches
    1 + 2r.  The nodes lie on the degree-4 interpolant of the sphere, within about 1e-4 of it."""
    from synth import real_ylm

    s = sphere80
    T = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, s.tgt_xyz, n_max=10 ** 6, t_f=TF)
    L = O.build_lists(T)
    R = T.root_radius
    assert T.n_boxes == 1 and np.all(T.root_center == 0.0) and R == 2.0 ** round(np.log2(R))
    f = O.center_features(T, L, s.src_w, real_ylm(2, 1, s.src_xyz), None, s.src_n, s.ctr_xyz, s.ctr_r)
    inside = np.linalg.norm(s.ctr_xyz, axis=0) < 1.0
    assert inside.sum() == s.n_ctr // 2
    assert np.allclose(f[inside, 2], 1.0 / R, atol=2e-4 / R)
    assert np.allclose(f[~inside, 2], (1.0 + 2.0 * s.ctr_r[~inside]) / R, atol=2e-4 / R)
    assert np.all(f[:, 1] == 0.0)
    assert np.allclose(2.0 ** f[:, 0] * R, s.ctr_r, rtol=1e-6)
    assert np.allclose(f[:, 3], 0.0, atol=1e-6)  # one box: its List 1 holds every source


def test_center_features_invariants(star_small):
    from synth import greens_density

    s = star_small
    u, dudn = greens_density(s)
    T = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, s.tgt_xyz, n_max=16, t_f=TF)
    L = O.build_lists(T)
    f = O.center_features(T, L, s.src_w, dudn, -u, s.src_n, s.ctr_xyz, s.ctr_r)
    b = T.ctr_owner
    # features 0 and 1 together give r / |root|: |b| = |root| 2^-level
    assert np.allclose(2.0 ** (f[:, 0] - 8.0 * f[:, 1]) * T.root_radius, s.ctr_r, rtol=1e-5)
    assert np.all(8.0 * f[:, 1] == T.level[b])
    # a center owned by a box below the root lies in that box's target confinement region
    assert np.all(f[b > 0, 2] <= np.sqrt(3.0) * (1.0 + TF) * (1 + 1e-6))
    assert np.all(f[:, 3] <= 1e-6)
    # a single nonzero source: centers whose List 1 holds its leaf see 0, every other center -12
    sig = np.zeros(s.n_src)
    j = 1234
    sig[j] = 1.0
    g = O.center_features(T, L, s.src_w, sig, None, s.src_n, s.ctr_xyz, s.ctr_r)
    hot = np.array([T.src_owner[j] in L.of("U", bb) for bb in b])
    assert hot.any() and not hot.all()
    assert np.allclose(g[hot, 3], 0.0, atol=1e-6) and np.allclose(g[~hot, 3], -12.0, atol=1e-5)


def test_fallback_raises_exactly_the_missing_targets(star_small):
    s = star_small
    vol = np.random.default_rng(8).uniform(-1.5, 1.5, size=(3, 30))
    t = np.concatenate([s.tgt_xyz, vol], axis=1)
    tc = np.concatenate([s.tgt_ctr, -np.ones(30, np.int32)]).astype(np.int32)
    T = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, t, n_max=16, t_f=TF)
    nt = t.shape[1]
    judge = np.linspace(-1.0, 1.0, nt)
    res = judge.copy()
    miss = [5, 77, s.n_ctr + 3]  # two QBX targets and one point target
    tol = 2.0 ** -20
    res[miss[0]] += 2 * tol
    res[miss[1]] = np.nan
    res[miss[2]] -= 5 * tol
    judge[9], res[9] = 0.5, 0.5 + tol  # exactly at the threshold: not a miss
    q = np.full(s.n_ctr, 3, np.int32)
    pb = np.full(T.n_boxes, 5, np.int32)
    n = O.orders_fallback(T, res, judge, tc, tol, 8, 16, q, pb)
    assert n == 3
    want_q = np.full(s.n_ctr, 3)
    want_p = np.full(T.n_boxes, 5)
    for t_ in miss:
        if tc[t_] >= 0:
            want_q[tc[t_]] = 8
            b = T.ctr_owner[tc[t_]]
        else:
            b = T.tgt_owner[t_]
        while b >= 0:
            want_p[b] = 16
            b = T.parent[b]
    assert np.array_equal(q, want_q) and np.array_equal(pb, want_p)
    assert pb[0] == 16 and np.sum(pb == 16) < T.n_boxes  # the root is on every chain; most boxes are not
