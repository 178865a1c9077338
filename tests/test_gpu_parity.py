"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

* Tree (Algorithm 4 Stage 1) and the six interaction lists (Section 5.2): bit-exact.
* Potentials of Algorithm 4 Stages 2-9 in FP64: normwise relative l-infinity error
  <= 1e-10 against the oracle's own Algorithm 4 on the same tree and lists.
"""
import numpy as np
import pytest

import oracle as O
from synth import greens_density, make_surface, real_ylm, star_radius
from synth.surfaces import STAR_Y63

from conftest import rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


def _cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


@pytest.fixture(scope="module")
def G():
    import paper_1805_06106_gb300 as G

    G.lib()
    return G


def _gpu_tree(G, s, tgt_xyz=None, n_max=32, t_f=0.9):
    t = s.tgt_xyz if tgt_xyz is None else tgt_xyz
    return G.qbx_build_tree(_cuda(s.src_xyz), _cuda(s.ctr_xyz), _cuda(s.ctr_r), _cuda(t), n_max=n_max, t_f=t_f)


def _assert_tree_equal(Tg, To):
    e = {k: v.cpu().numpy() for k, v in Tg.export().items()}
    assert Tg.n_boxes == To.n_boxes
    assert Tg.info.n_levels == To.n_levels
    assert np.array_equal(e["level"], To.level)
    assert np.array_equal(e["coords"], To.coords)
    assert np.array_equal(e["parent"], To.parent)
    assert np.array_equal(e["child"], To.child)
    for k in ("src_owner", "ctr_owner", "tgt_owner"):
        assert np.array_equal(e[k], getattr(To, k)), k
    assert list(Tg.info.root_center) == list(To.root_center) and Tg.info.root_radius == To.root_radius


@pytest.mark.parametrize("surf_name,n_max", [("sphere80", 8), ("sphere80", 32), ("star_small", 16),
                                             ("star_small", 64), ("sphere320", 32)])
def test_tree_and_lists_bit_exact(G, surf_name, n_max, request):
    s = request.getfixturevalue(surf_name)
    Tg = _gpu_tree(G, s, n_max=n_max)
    To = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, s.tgt_xyz, n_max=n_max, t_f=0.9)
    _assert_tree_equal(Tg, To)
    Lg = G.qbx_build_lists(Tg).export()
    Lo = O.build_lists(To)
    for name in O.LIST_NAMES:
        st, ix = (x.cpu().numpy() for x in Lg[name])
        assert np.array_equal(st, Lo.start[name]), name
        assert np.array_equal(ix, Lo.idx[name]), name


def test_tree_with_coincident_points_and_depth_cap(G):
    """All particles at two points: splitting stops at max_depth and the leaves stay overfull."""
    rng = np.random.default_rng(0)
    pts = np.repeat(np.array([[0.1, 0.2, 0.3], [0.1000001, 0.2, 0.3]]).T, 40, axis=1)
    ctr = pts + 1e-3
    r = np.full(ctr.shape[1], 1e-4)
    Tg = G.qbx_build_tree(_cuda(pts), _cuda(ctr), _cuda(r), _cuda(pts), n_max=8, t_f=0.9, max_depth=12)
    To = O.build_tree(pts, ctr, r, pts, n_max=8, t_f=0.9, max_depth=12)
    _assert_tree_equal(Tg, To)
    assert Tg.info.n_overfull == To.n_overfull > 0
    del rng


def _eval_both(G, s, sigma, mu, tgt_xyz, tgt_ctr, p_qbx, p_fmm, n_max=32, qctr=None, pbox=None):
    Tg = _gpu_tree(G, s, tgt_xyz=tgt_xyz, n_max=n_max)
    Lg = G.qbx_build_lists(Tg)
    pot = G.qbx_eval(Tg, Lg, _cuda(s.src_w), None if sigma is None else _cuda(sigma),
                     None if mu is None else _cuda(mu), _cuda(s.src_n), _cuda(tgt_ctr, torch.int32), p_qbx, p_fmm,
                     p_qbx_per_ctr=None if qctr is None else _cuda(qctr, torch.int8),
                     p_fmm_per_box=None if pbox is None else _cuda(pbox, torch.int8)).cpu().numpy()
    To = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, tgt_xyz, n_max=n_max, t_f=0.9)
    Lo = O.build_lists(To)
    ref = O.fmm_eval(To, Lo, s.src_xyz, s.src_w, sigma, mu, s.src_n, s.ctr_xyz, tgt_xyz, tgt_ctr, p_qbx, p_fmm,
                     p_qbx_ctr=qctr, p_fmm_box=pbox)
    return pot, ref, (Tg, Lg)


@pytest.mark.parametrize("p_qbx,p_fmm", [(5, 10), (3, 4), (7, 15), (8, 16)])
def test_single_layer_parity_sphere(G, sphere80, p_qbx, p_fmm):
    s = sphere80
    sig = real_ylm(2, 1, s.src_xyz)
    pot, ref, _ = _eval_both(G, s, sig, None, s.tgt_xyz, s.tgt_ctr, p_qbx, p_fmm)
    assert rel_linf(pot, ref) <= TOL_FP64


@pytest.mark.parametrize("p_qbx,p_fmm,n_max", [(5, 8, 32), (7, 12, 16), (12, 16, 64)])
def test_single_and_double_layer_with_point_targets(G, star_small, p_qbx, p_fmm, n_max):
    s = star_small
    u, dudn = greens_density(s)
    rng = np.random.default_rng(11)
    vol = rng.uniform(-2.0, 2.0, size=(3, 400))
    t = np.concatenate([s.tgt_xyz, vol], axis=1)
    tc = np.concatenate([s.tgt_ctr, -np.ones(400, np.int32)]).astype(np.int32)
    pot, ref, _ = _eval_both(G, s, dudn, -u, t, tc, p_qbx, p_fmm, n_max=n_max)
    assert rel_linf(pot, ref) <= TOL_FP64
    # point targets alone, normwise over themselves
    assert rel_linf(pot[s.n_ctr:], ref[s.n_ctr:]) <= TOL_FP64


def test_double_layer_only_and_all_point_targets(G, sphere80):
    s = sphere80
    mu = real_ylm(3, -2, s.src_xyz)
    tc = -np.ones(s.n_ctr, np.int32)
    tgt = s.ctr_xyz.copy()  # off-surface points evaluated by plain quadrature
    pot, ref, _ = _eval_both(G, s, None, mu, tgt, tc, 4, 8)
    assert rel_linf(pot, ref) <= TOL_FP64


def test_per_center_and_per_box_orders(G, star_small):
    s = star_small
    sig = random_density = real_ylm(4, 1, s.src_xyz) + 0.3
    del random_density
    Tg = _gpu_tree(G, s)
    rng = np.random.default_rng(5)
    qctr = rng.integers(2, 9, s.n_ctr).astype(np.int8)
    pbox = rng.integers(6, 13, Tg.n_boxes).astype(np.int8)
    pot, ref, _ = _eval_both(G, s, sig, None, s.tgt_xyz, s.tgt_ctr, 8, 12, qctr=qctr, pbox=pbox)
    assert rel_linf(pot, ref) <= TOL_FP64


def test_repeat_is_bitwise_deterministic(G, star_small):
    s = star_small
    u, dudn = greens_density(s)
    Tg = _gpu_tree(G, s)
    Lg = G.qbx_build_lists(Tg)
    args = (_cuda(s.src_w), _cuda(dudn), _cuda(-u), _cuda(s.src_n), _cuda(s.tgt_ctr, torch.int32), 7, 15)
    a = G.qbx_eval(Tg, Lg, *args).cpu().numpy()
    b = G.qbx_eval(Tg, Lg, *args).cpu().numpy()
    assert np.array_equal(a, b)


def test_invalid_arguments_are_reported(G, sphere80):
    s = sphere80
    Tg = _gpu_tree(G, s)
    Lg = G.qbx_build_lists(Tg)
    w, sig, n = _cuda(s.src_w), _cuda(real_ylm(1, 0, s.src_xyz)), _cuda(s.src_n)
    tc = _cuda(s.tgt_ctr, torch.int32)
    with pytest.raises(G.QbxError) as e:
        G.qbx_eval(Tg, Lg, w, sig, None, n, tc, 9, 8)  # p_qbx > p_fmm
    assert e.value.code == -1
    with pytest.raises(G.QbxError) as e:
        G.qbx_eval(Tg, Lg, w, sig, None, n, tc, 5, 25)
    assert e.value.code == -1
    bad = tc.clone()
    bad[3] = s.n_ctr + 7
    with pytest.raises(G.QbxError) as e:
        G.qbx_eval(Tg, Lg, w, sig, None, n, bad, 5, 10)
    assert e.value.code == -1
    wbad = w.clone()
    wbad[0] = float("nan")
    with pytest.raises(G.QbxError):
        G.qbx_eval(Tg, Lg, wbad, sig, None, n, tc, 5, 10)
    x = _cuda(s.src_xyz)
    x[1, 5] = float("inf")
    with pytest.raises(G.QbxError) as e:
        G.qbx_build_tree(x, _cuda(s.ctr_xyz), _cuda(s.ctr_r), _cuda(s.tgt_xyz))
    assert e.value.code == -1
    r = _cuda(s.ctr_r)
    r[0] = 0.0
    with pytest.raises(G.QbxError):
        G.qbx_build_tree(_cuda(s.src_xyz), _cuda(s.ctr_xyz), r, _cuda(s.tgt_xyz))
    # the library is still usable afterwards
    pot = G.qbx_eval(Tg, Lg, w, sig, None, n, tc, 5, 10)
    assert torch.isfinite(pot).all()


def test_no_sources_gives_zero(G):
    s = make_surface(1, star_radius(STAR_Y63))
    empty = np.zeros((3, 0))
    Tg = G.qbx_build_tree(_cuda(empty), _cuda(s.ctr_xyz), _cuda(s.ctr_r), _cuda(s.tgt_xyz))
    Lg = G.qbx_build_lists(Tg)
    z = torch.zeros(0, dtype=torch.float64, device="cuda")
    pot = G.qbx_eval(Tg, Lg, z, z, None, torch.zeros((3, 0), dtype=torch.float64, device="cuda"),
                     _cuda(s.tgt_ctr, torch.int32), 5, 10)
    assert torch.count_nonzero(pot) == 0


def test_stage_profiling_leaves_results_unchanged(G, star_small):
    """Per-stage event timing changes no result; the stages that only the mixed-precision modes
    fill (List 3 far products and their reduction) are empty in FP64."""
    s = star_small
    u, dudn = greens_density(s)
    Tg = _gpu_tree(G, s)
    Lg = G.qbx_build_lists(Tg)
    args = (_cuda(s.src_w), _cuda(dudn), _cuda(-u), _cuda(s.src_n), _cuda(s.tgt_ctr, torch.int32), 7, 15)
    for prec in (G.QBX_FP64, G.QBX_M2L_3XTF32):
        Lg.profile(False)
        a = G.qbx_eval(Tg, Lg, *args, precision=prec).cpu().numpy()
        Lg.profile(True)
        b = G.qbx_eval(Tg, Lg, *args, precision=prec).cpu().numpy()
        ms = Lg.stage_ms()
        Lg.profile(False)
        assert np.array_equal(a, b)
        assert tuple(ms) == G.STAGE_NAMES and len(ms) == 10
        assert all(v >= 0.0 for v in ms.values())
        assert ms["centers"] > 0.0
        if prec == G.QBX_FP64:
            assert ms["m2qbxl_mixed"] < 0.05 and ms["m2qbxl_reduce"] < 0.05


def test_order_sweep_columns_match_oracle_at_each_order(G, sphere80):
    """Column q of qbx_eval_order_sweep is the evaluation with p_qbx = q (same p_fmm): against the oracle
    at q = 0, 2 and the full order, double layer, with point targets (1e-10)."""
    s = sphere80
    u, dudn = greens_density(s)
    vol = np.random.default_rng(4).uniform(-1.6, 1.6, size=(3, 60))
    t = np.concatenate([s.tgt_xyz, vol], axis=1)
    tc = np.concatenate([s.tgt_ctr, -np.ones(60, np.int32)]).astype(np.int32)
    Q, P = 6, 10
    T = G.qbx_build_tree(_cuda(s.src_xyz), _cuda(s.ctr_xyz), _cuda(s.ctr_r), _cuda(t), n_max=16, t_f=0.9)
    L = G.qbx_build_lists(T)
    part = G.qbx_eval_order_sweep(T, L, _cuda(s.src_w), _cuda(dudn), _cuda(-u), _cuda(s.src_n),
                                  _cuda(tc, torch.int32), Q, P).cpu().numpy()
    To = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, t, n_max=16, t_f=0.9)
    Lo = O.build_lists(To)
    for q in (0, 2, Q):
        ref = O.fmm_eval(To, Lo, s.src_xyz, s.src_w, dudn, -u, s.src_n, s.ctr_xyz, t, tc, q, P)
        assert rel_linf(part[q], ref) <= 1e-10, q
