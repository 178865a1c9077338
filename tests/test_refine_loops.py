"""The stage-1 and stage-2 refinement loops (Algorithms 1 and 2, Sections 3.2-3.3) on the host,
driven here by the oracle's element marks instead of the GPU's (no GPU): on two unit spheres 0.03
apart the loops end, each leaves nothing for the oracle to mark, stage 1 refines only the elements
near the gap (the far hemispheres keep their size), and stage 2 never moves a center."""
import numpy as np

import oracle as O
from paper_1805_06106_gb300 import refine
from synth import bisect_flat, flat_mesh, scaled_curvature

from conftest import two_spheres


def _oracle_marks(d, which, eps):
    elem = d.ctr_elem if which == 0 else d.src_elem
    return O.refine_marks(which, d.src_xyz, d.ctr_xyz, d.ctr_r, elem, d.n_elem, d.elem_eta, eps=eps)


def _bisect(ms, marks):
    offs = np.cumsum([0] + [len(m) for m in ms])[:-1]
    return [bisect_flat(m, marks[o:o + len(m)]) for m, o in zip(ms, offs)]


def test_refinement_loops_on_two_close_spheres():
    gap = 0.03
    m0 = [flat_mesh(2), flat_mesh(2)]
    curv = lambda ms: np.concatenate([scaled_curvature(m) for m in ms])  # noqa: E731
    m1, d1, hist1 = refine.stage1(m0, lambda ms: two_spheres(ms, gap), _bisect, curvature=curv,
                                  marks_fn=_oracle_marks)
    assert hist1[0] > 0 and hist1[-1] == 0
    assert not _oracle_marks(d1, 0, refine.EPS_DISTURB).any()
    # only elements near the gap were refined: the smallest elements face the other sphere
    for m, sign in zip(m1, (1.0, -1.0)):
        cen = m.mean(axis=1)
        area = 0.5 * np.linalg.norm(np.cross(m[:, 1] - m[:, 0], m[:, 2] - m[:, 0]), axis=1)
        near = sign * cen[:, 0] > 0.5
        assert area[near].min() < area[~near].min() / 3.0
        assert np.allclose(area[sign * cen[:, 0] < -0.5], area[sign * cen[:, 0] < -0.5].max(), rtol=0.5)
    m2, d2, hist2 = refine.stage2(m1, lambda a, b: two_spheres(a, gap, b), _bisect, marks_fn=_oracle_marks)
    assert hist2[-1] == 0
    assert not _oracle_marks(d2, 1, refine.EPS_DISTURB).any()
    assert np.array_equal(d2.ctr_xyz, d1.ctr_xyz) and np.array_equal(d2.ctr_r, d1.ctr_r)
    assert d2.n_elem >= d1.n_elem
