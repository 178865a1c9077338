"""The interior Dirichlet solve with the GPU evaluation as the operator (paper_1805_06106_gb300.solve):
GMRES on D^-[mu] = f through qbx_eval converges, and the double-layer potential of the solved density,
evaluated by qbx_eval at point targets inside the sphere, reproduces the harmonic function 1/|x - x0|."""
import numpy as np
import pytest

from synth import collocation_surface, flat_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cu(a, dt=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dt is None else t.to(dt)).cuda()


def test_interior_dirichlet_on_the_gpu():
    import paper_1805_06106_gb300 as G
    from paper_1805_06106_gb300.solve import interior_dirichlet, interpolate

    s = collocation_surface(flat_mesh(2))
    n = s.n_ctr // 2
    nodes = s.tgt_xyz[:, :n]
    x0 = np.array([3.0, 1.0, 2.0])
    T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(nodes), n_max=32)
    L = G.qbx_build_lists(T)
    w, nrm, interp = _cu(s.src_w), _cu(s.src_n), _cu(s.interp)
    f = _cu(1.0 / np.linalg.norm(nodes - x0[:, None], axis=0))
    mu, info = interior_dirichlet(T, L, w, nrm, _cu(np.arange(n, 2 * n), torch.int32), interp, f, 5, 10, tol=1e-4,
                                  restart=80, maxiter=200)
    assert info["converged"] and info["iterations"] < 60
    pts = np.random.default_rng(4).normal(size=(3, 64))
    pts *= 0.5 / np.linalg.norm(pts, axis=0)
    T2 = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(pts), n_max=32)
    L2 = G.qbx_build_lists(T2)
    u = G.qbx_eval(T2, L2, w, None, interpolate(interp, mu), nrm, _cu(-np.ones(64), torch.int32), 5, 10)
    exact = 1.0 / np.linalg.norm(pts - x0[:, None], axis=0)
    assert np.max(np.abs(u.cpu().numpy() - exact)) / np.max(exact) < 1e-4
