"""Tree variants and per-stage precision through the C ABI, against the CPU oracle.

* QBX_TREE_LINF_TCR (the box-shaped TCR of Table l2-comparison's left columns) and
  QBX_TREE_LEVEL_RESTRICT (Section 5.3, Remark on level restriction), alone and together:
  tree arrays and the six lists bit for bit, qbx_lists_cost exactly, and FP64 potentials on the
  variant trees within 1e-10 of the oracle's Algorithm 4 on the same tree.
* QBX_MIXED_M2L_ONLY / QBX_MIXED_M2QBXL_ONLY: each reduced-precision stage on its own within
  1e-6 of the oracle, so the error of List 2 M2L and of List 3 far M2QBXL is known separately.
"""
import numpy as np
import pytest

import oracle as O
from synth import greens_density, real_ylm

from conftest import rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARIANTS = [(True, False), (False, True), (True, True)]


def _cu(a, dt=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dt is None else t.to(dt)).cuda()


@pytest.fixture(scope="module")
def G():
    import paper_1805_06106_gb300 as G

    G.lib()
    return G


def _pair(G, s, t, n_max, linf, restrict):
    Tg = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(t), n_max=n_max, t_f=0.9,
                          linf_tcr=linf, level_restrict=restrict)
    To = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, t, n_max=n_max, t_f=0.9, linf_tcr=linf,
                      level_restrict=restrict)
    return Tg, To


def _assert_tree_equal(Tg, To):
    e = {k: v.cpu().numpy() for k, v in Tg.export().items()}
    assert Tg.n_boxes == To.n_boxes
    assert Tg.info.n_levels == To.n_levels
    for k in ("level", "coords", "parent", "child"):
        assert np.array_equal(e[k], getattr(To, k)), k
    for k in ("src_owner", "ctr_owner", "tgt_owner"):
        assert np.array_equal(e[k], getattr(To, k)), k
    assert Tg.info.n_overfull == To.n_overfull


@pytest.mark.parametrize("linf,restrict", VARIANTS)
@pytest.mark.parametrize("surf_name,n_max", [("sphere80", 8), ("star_small", 8), ("star_small", 32),
                                             ("sphere320", 16)])
def test_variant_tree_lists_cost_bit_exact(G, surf_name, n_max, linf, restrict, request):
    s = request.getfixturevalue(surf_name)
    Tg, To = _pair(G, s, s.tgt_xyz, n_max, linf, restrict)
    _assert_tree_equal(Tg, To)
    Lg = G.qbx_build_lists(Tg)
    Lo = O.build_lists(To)
    ex = Lg.export()
    for name in O.LIST_NAMES:
        st, ix = (x.cpu().numpy() for x in ex[name])
        assert np.array_equal(st, Lo.start[name]), name
        assert np.array_equal(ix, Lo.idx[name]), name
    got = G.qbx_lists_cost(Lg, 5, 15)
    want = O.lists_cost(To, Lo, 5, 15)
    assert got["count"] == O.lists_counts(To, Lo)
    for k in O.LIST_NAMES:
        assert got["ops"][k] == want[k], k
    assert got["total"] == want["total"]


def test_level_restriction_of_a_tree_that_is_already_restricted(G):
    """A regular lattice of sources: every leaf on one level, so the flag changes nothing."""
    g = (np.arange(8) + 0.5) / 8.0
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    src = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    e = np.zeros((3, 0))
    T0 = G.qbx_build_tree(_cu(src), _cu(e), _cu(np.zeros(0)), _cu(e), n_max=1)
    T1 = G.qbx_build_tree(_cu(src), _cu(e), _cu(np.zeros(0)), _cu(e), n_max=1, level_restrict=True)
    a, b = T0.export(), T1.export()
    for k in ("level", "coords", "parent", "child", "src_owner"):
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("linf,restrict", VARIANTS)
def test_variant_fp64_potentials(G, star_small, linf, restrict):
    s = star_small
    u, dudn = greens_density(s)
    rng = np.random.default_rng(7)
    vol = rng.uniform(-2.0, 2.0, size=(3, 200))
    t = np.concatenate([s.tgt_xyz, vol], axis=1)
    tc = np.concatenate([s.tgt_ctr, -np.ones(200, np.int32)]).astype(np.int32)
    Tg, To = _pair(G, s, t, 16, linf, restrict)
    Lg = G.qbx_build_lists(Tg)
    pot = G.qbx_eval(Tg, Lg, _cu(s.src_w), _cu(dudn), _cu(-u), _cu(s.src_n), _cu(tc, torch.int32), 7, 12)
    ref = O.fmm_eval(To, O.build_lists(To), s.src_xyz, s.src_w, dudn, -u, s.src_n, s.ctr_xyz, t, tc, 7, 12)
    assert rel_linf(pot.cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("form", ["fp32", "3xtf32"])
def test_each_reduced_precision_stage_alone(G, star_small, form):
    s = star_small
    sig = real_ylm(3, 2, s.src_xyz)
    base = {"fp32": G.QBX_M2L_FP32, "3xtf32": G.QBX_M2L_3XTF32}[form]
    T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(s.tgt_xyz), n_max=32, t_f=0.9)
    L = G.qbx_build_lists(T)
    args = (_cu(s.src_w), _cu(sig), None, _cu(s.src_n), _cu(s.tgt_ctr, torch.int32), 7, 15)
    To = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, s.tgt_xyz, n_max=32, t_f=0.9)
    ref = O.fmm_eval(To, O.build_lists(To), s.src_xyz, s.src_w, sig, None, s.src_n, s.ctr_xyz, s.tgt_xyz,
                     s.tgt_ctr, 7, 15)
    out = {}
    for name, prec in (("fp64", G.QBX_FP64), ("both", base), ("m2l", base | G.QBX_MIXED_M2L_ONLY),
                       ("m2qbxl", base | G.QBX_MIXED_M2QBXL_ONLY)):
        out[name] = G.qbx_eval(T, L, *args, precision=prec).cpu().numpy()
    assert rel_linf(out["fp64"], ref) <= 1e-10
    for name in ("both", "m2l", "m2qbxl"):
        err = rel_linf(out[name], ref)
        assert 1e-14 < err <= 1e-6, (name, err)  # reduced precision ran, within the mixed tolerance
    # each single-stage result differs from the two-stage one: the other stage really was FP64
    assert not np.array_equal(out["m2l"], out["both"]) and not np.array_equal(out["m2qbxl"], out["both"])
    again = G.qbx_eval(T, L, *args, precision=base | G.QBX_MIXED_M2QBXL_ONLY).cpu().numpy()
    assert np.array_equal(again, out["m2qbxl"])


def test_stage_selection_needs_a_reduced_mode(G, sphere80):
    s = sphere80
    sig = real_ylm(2, 1, s.src_xyz)
    T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(s.tgt_xyz), n_max=32)
    L = G.qbx_build_lists(T)
    args = (_cu(s.src_w), _cu(sig), None, _cu(s.src_n), _cu(s.tgt_ctr, torch.int32), 5, 10)
    for bad in (G.QBX_MIXED_M2L_ONLY, G.QBX_M2L_FP32 | G.QBX_MIXED_M2L_ONLY | G.QBX_MIXED_M2QBXL_ONLY,
                G.QBX_M2L_3XTF32 | 0x40):
        with pytest.raises(G.QbxError):
            G.qbx_eval(T, L, *args, precision=bad)
