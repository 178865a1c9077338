"""Element marks of Algorithms 1 and 2 (Section 3) on the GPU against the oracle's definitions
(bit for bit), and the stage-1 / stage-2 refinement loops built on them: they finish, the oracle
finds nothing left to mark on their output, and stage-1 refinement repairs the QBX error that
interfering geometry causes (Green's formula on two nearly touching spheres)."""
import numpy as np
import pytest

import oracle as O
from synth import bisect_flat, flat_mesh, scaled_curvature, star_radius, surface_from_flat

from conftest import rel_linf, two_spheres as _two_spheres

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cu(a, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()


def _gpu_marks(import_G, d, which, n_max):
    G = import_G
    T = G.qbx_build_tree(_cu(d.src_xyz), _cu(d.ctr_xyz), _cu(d.ctr_r), _cu(np.zeros((3, 0))), n_max=n_max)
    if which == G.QBX_REFINE_INTERFERING:
        m = G.qbx_refine_marks(T, which, _cu(d.ctr_elem, torch.int32), d.n_elem, eps=0.025)
    else:
        m = G.qbx_refine_marks(T, which, _cu(d.src_elem, torch.int32), d.n_elem, elem_eta=_cu(d.elem_eta))
    return m.cpu().numpy().astype(bool)


@pytest.fixture(scope="module")
def G():
    import paper_1805_06106_gb300 as G

    G.lib()
    return G


@pytest.mark.parametrize("gap", [0.02, 0.08, 0.5])
@pytest.mark.parametrize("n_max", [8, 64])
def test_interfering_marks_match_oracle(G, gap, n_max):
    d = _two_spheres([flat_mesh(4), flat_mesh(3)], gap)
    got = _gpu_marks(G, d, G.QBX_REFINE_INTERFERING, n_max)
    want = O.refine_marks(0, d.src_xyz, d.ctr_xyz, d.ctr_r, d.ctr_elem, d.n_elem, eps=0.025)
    assert np.array_equal(got, want)
    assert (gap < 0.1) == bool(want.any())


@pytest.mark.parametrize("n_max", [8, 64])
def test_quadrature_marks_match_oracle(G, n_max):
    f = flat_mesh(4)
    bis = np.zeros(len(f), bool)
    bis[[3, 40, 41, 200]] = True
    f1 = bisect_flat(f, bis)
    d = _two_spheres([f1, flat_mesh(3)], 0.05)
    got = _gpu_marks(G, d, G.QBX_REFINE_QUAD_RES, n_max)
    want = O.refine_marks(1, d.src_xyz, d.ctr_xyz, d.ctr_r, d.src_elem, d.n_elem, d.elem_eta)
    assert np.array_equal(got, want) and want.any()


def test_marks_on_a_star(G):
    s = surface_from_flat(flat_mesh(6), star_radius([(0.4, 8, 4)]))
    for which, elem in ((G.QBX_REFINE_INTERFERING, s.ctr_elem), (G.QBX_REFINE_QUAD_RES, s.src_elem)):
        got = _gpu_marks(G, s, which, 32)
        want = O.refine_marks(which, s.src_xyz, s.ctr_xyz, s.ctr_r, elem, s.n_elem, s.elem_eta)
        assert np.array_equal(got, want)


def test_refinement_loops_and_their_effect(G):
    """Two unit spheres 0.03 apart at a coarse resolution: the exterior expansion balls facing the gap
    hold the other sphere's sources.  Stage-1 refinement bisects until none does; stage 2 then
    refines the source mesh; on each result the oracle marks nothing.  Green's formula
    S(d_n u) - D(u) = u/2 (u = 1/|x - x0| with x0 outside both spheres) shows the repair."""
    from paper_1805_06106_gb300 import refine

    gap = 0.03
    m0 = [flat_mesh(2), flat_mesh(2)]
    disc = lambda ms: _two_spheres(ms, gap)  # noqa: E731
    bis = lambda ms, marks: [bisect_flat(m, marks[o:o + len(m)])  # noqa: E731
                             for m, o in zip(ms, np.cumsum([0] + [len(x) for x in ms])[:-1])]
    curv = lambda ms: np.concatenate([scaled_curvature(m) for m in ms])  # noqa: E731
    m1, d1, hist1 = refine.stage1(m0, disc, bis, curvature=curv)
    assert hist1[0] > 0 and hist1[-1] == 0 and len(hist1) >= 2
    assert not O.refine_marks(0, d1.src_xyz, d1.ctr_xyz, d1.ctr_r, d1.ctr_elem, d1.n_elem, eps=0.025).any()
    m2, d2, hist2 = refine.stage2(m1, lambda a, b: _two_spheres(a, gap, b), bis)
    assert hist2[-1] == 0
    assert not O.refine_marks(1, d2.src_xyz, d2.ctr_xyz, d2.ctr_r, d2.src_elem, d2.n_elem, d2.elem_eta).any()
    assert d2.n_elem >= d1.n_elem

    x0 = np.array([-0.5, 3.0, 1.0])

    def greens_error(d):
        r = d.src_xyz - x0[:, None]
        dist = np.linalg.norm(r, axis=0)
        u, dudn = 1.0 / dist, -np.sum(r * d.src_n, axis=0) / dist ** 3
        T = G.qbx_build_tree(_cu(d.src_xyz), _cu(d.ctr_xyz), _cu(d.ctr_r), _cu(d.tgt_xyz), n_max=32)
        L = G.qbx_build_lists(T)
        pot = G.qbx_eval(T, L, _cu(d.src_w), _cu(dudn), _cu(-u), _cu(d.src_n), _cu(d.tgt_ctr, torch.int32), 8, 16)
        pot = pot.cpu().numpy()
        ut = 1.0 / np.linalg.norm(d.tgt_xyz - x0[:, None], axis=0)
        # the average of the exterior and interior limits of each node is u/2
        parts, i0 = [], 0
        for p in d.parts:
            n = p.n_ctr // 2
            parts.append(0.5 * (pot[i0:i0 + n] + pot[i0 + n:i0 + 2 * n]) - 0.5 * ut[i0:i0 + n])
            i0 += 2 * n
        return float(np.max(np.abs(np.concatenate(parts)))) / float(np.max(np.abs(ut)))

    e0 = greens_error(_two_spheres(m0, gap))
    e1 = greens_error(d1)
    e2 = greens_error(d2)
    assert e1 < 0.2 * e0, (e0, e1, e2)
    assert e2 <= 1.5 * e1, (e0, e1, e2)
