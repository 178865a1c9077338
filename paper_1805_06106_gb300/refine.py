"""Geometry processing of Section 3 driven by the library's element marks (qbx_refine_marks).

Stage-1 refinement (Section 3.2): Algorithm 1 bisects every element whose expansion balls are
disturbed by source geometry, together with the scaled-curvature criterion (eq.
curvature-criterion, kappa_k <= 0.8), until nothing is marked.  Stage-2 refinement (Section 3.3):
Algorithm 2 bisects source elements of a second mesh, starting from the stage-1 mesh, until no
expansion center lies within 0.5 (3/4) eta of a source of a coarser element; centers and radii
stay those of stage 1.  Each round builds a tree of the sources and centers on the GPU and marks
on the GPU; the caller owns the mesh and supplies how to discretize and bisect it.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B

EPS_DISTURB = 0.025   # Algorithm 1's tolerance that keeps a center's own source point out of its test
KAPPA_MAX = 0.8       # scaled-curvature threshold (Section 3.2.1)


def _tree(src_xyz, ctr_xyz, ctr_r, n_max):
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()  # noqa: E731
    empty = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    return B.qbx_build_tree(cu(src_xyz), cu(ctr_xyz), cu(ctr_r), empty, n_max=n_max)


def gpu_marks(d, which, eps=EPS_DISTURB, n_max=64):
    """Element marks of one discretization on the GPU: a tree of its sources and centers, then
    qbx_refine_marks (which = QBX_REFINE_INTERFERING or QBX_REFINE_QUAD_RES).  bool[n_elem] on the host."""
    T = _tree(d.src_xyz, d.ctr_xyz, d.ctr_r, n_max)
    if which == B.QBX_REFINE_INTERFERING:
        ce = torch.from_numpy(np.ascontiguousarray(d.ctr_elem, np.int32)).cuda()
        m = B.qbx_refine_marks(T, which, ce, d.n_elem, eps=eps)
    else:
        se = torch.from_numpy(np.ascontiguousarray(d.src_elem, np.int32)).cuda()
        eta = torch.from_numpy(np.ascontiguousarray(d.elem_eta, np.float64)).cuda()
        m = B.qbx_refine_marks(T, which, se, d.n_elem, elem_eta=eta)
    return m.cpu().numpy().astype(bool)


def stage1(mesh, discretize, bisect, curvature=None, eps=EPS_DISTURB, kappa_max=KAPPA_MAX, n_max=64,
           max_rounds=16, marks_fn=None):
    """Algorithm 1 (+ the scaled-curvature criterion when `curvature(mesh)` gives kappa per element).
    discretize(mesh) -> object with src_xyz, ctr_xyz, ctr_r, ctr_elem (element of each center) and
    n_elem; bisect(mesh, marks) -> refined mesh; marks_fn(d, which, eps) replaces the GPU marks
    (gpu_marks) when given.  Returns (mesh, discretization, marked per round)."""
    history = []
    for _ in range(max_rounds):
        d = discretize(mesh)
        marks = (marks_fn(d, B.QBX_REFINE_INTERFERING, eps) if marks_fn else
                 gpu_marks(d, B.QBX_REFINE_INTERFERING, eps, n_max))
        if curvature is not None:
            marks |= np.asarray(curvature(mesh)) > kappa_max
        history.append(int(marks.sum()))
        if not marks.any():
            return mesh, d, history
        mesh = bisect(mesh, marks)
    raise RuntimeError(f"stage-1 refinement still marking after {max_rounds} rounds: {history}")


def stage2(mesh1, discretize2, bisect, n_max=64, max_rounds=16, marks_fn=None):
    """Algorithm 2 from the stage-1 mesh.  discretize2(mesh1, mesh2) -> object with the sources of
    mesh2 (src_xyz, src_elem, elem_eta, n_elem) and the centers of mesh1 (ctr_xyz, ctr_r); marks_fn as
    in stage1.  Returns (stage-2 mesh, discretization, marked per round)."""
    mesh2 = mesh1
    history = []
    for _ in range(max_rounds):
        d = discretize2(mesh1, mesh2)
        marks = (marks_fn(d, B.QBX_REFINE_QUAD_RES, EPS_DISTURB) if marks_fn else
                 gpu_marks(d, B.QBX_REFINE_QUAD_RES, n_max=n_max))
        history.append(int(marks.sum()))
        if not marks.any():
            return mesh2, d, history
        mesh2 = bisect(mesh2, marks)
    raise RuntimeError(f"stage-2 refinement still marking after {max_rounds} rounds: {history}")
