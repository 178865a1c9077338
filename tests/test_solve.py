"""The GMRES driver of the boundary-value solve (no GPU; the oracle's direct QBX stands in for the
evaluation as the operator).

* GMRES against a dense direct solve on seeded well-conditioned systems, with and without restarts.
* The interior Dirichlet problem for Laplace's equation as a double-layer potential (the use of
  Section 6.2): densities of degree 4 per element at interior collocation nodes, sources at a
  degree-10 stage-2 rule.  The solved density reproduces the harmonic function 1/|x - x0| (x0
  outside) and the constant 1 at points inside the sphere.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1805_06106_gb300.solve import dirichlet_double_layer, gmres
from synth import collocation_surface, flat_mesh


@pytest.mark.parametrize("restart", [200, 7])
def test_gmres_matches_a_direct_solve(restart):
    rng = np.random.default_rng(1)
    n = 120
    A = np.eye(n) * 2.0 + rng.normal(size=(n, n)) / np.sqrt(n) * 0.6
    b = rng.normal(size=n)
    At = torch.from_numpy(A)
    x, info = gmres(lambda v: At @ v, torch.from_numpy(b), tol=1e-12, restart=restart, maxiter=2000)
    assert info["converged"] and info["residuals"][-1] <= 1e-11
    ref = np.linalg.solve(A, b)
    assert np.max(np.abs(x.numpy() - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.fixture(scope="module")
def sphere_dirichlet():
    s = collocation_surface(flat_mesh(1))
    n = s.n_ctr // 2
    nodes = s.tgt_xyz[:, :n]
    tc = np.arange(n, 2 * n, dtype=np.int32)  # every node through its interior center

    def apply(mu_src):
        return torch.from_numpy(O.direct_eval(s.src_xyz, s.src_w, None, mu_src.numpy(), s.src_n, s.ctr_xyz, nodes,
                                              tc, 5))
    return s, nodes, apply, torch.from_numpy(s.interp)


def test_interior_dirichlet_reproduces_a_harmonic_function(sphere_dirichlet):
    s, nodes, apply, interp = sphere_dirichlet
    x0 = np.array([3.0, 1.0, 2.0])
    f = torch.from_numpy(1.0 / np.linalg.norm(nodes - x0[:, None], axis=0))
    mu, info = dirichlet_double_layer(apply, interp, f, tol=1e-4, restart=80, maxiter=200)
    assert info["converged"] and info["iterations"] < 40 and info["residuals"][-1] < 1e-4
    rng = np.random.default_rng(4)
    pts = rng.normal(size=(3, 50))
    pts *= 0.5 / np.linalg.norm(pts, axis=0)  # inside, clear of the surface: plain quadrature
    mu_src = (mu.numpy().reshape(-1, 15) @ s.interp.T).reshape(-1)
    u = O.direct_eval(s.src_xyz, s.src_w, None, mu_src, s.src_n, s.ctr_xyz, pts, -np.ones(50, np.int32), 5)
    exact = 1.0 / np.linalg.norm(pts - x0[:, None], axis=0)
    assert np.max(np.abs(u - exact)) / np.max(np.abs(exact)) < 1e-4


def test_constant_boundary_values(sphere_dirichlet):
    """f = 1 on the surface: u = 1 inside (the density itself is -1 up to the operator's near-null
    directions, which leave the potential unchanged)."""
    s, nodes, apply, interp = sphere_dirichlet
    mu, info = dirichlet_double_layer(apply, interp, torch.ones(nodes.shape[1], dtype=torch.float64), tol=1e-4,
                                      restart=80, maxiter=200)
    assert info["converged"]
    pts = np.random.default_rng(5).normal(size=(3, 40))
    pts *= 0.5 / np.linalg.norm(pts, axis=0)
    mu_src = (mu.numpy().reshape(-1, 15) @ s.interp.T).reshape(-1)
    u = O.direct_eval(s.src_xyz, s.src_w, None, mu_src, s.src_n, s.ctr_xyz, pts, -np.ones(40, np.int32), 5)
    assert np.max(np.abs(u - 1.0)) < 1e-4


@pytest.mark.parametrize("n,m", [(2, 1), (3, -2)])
def test_single_layer_normal_derivative_on_the_sphere(n, m):
    """S'[Y_n^m] on the unit sphere: the exterior limit is -(n+1)/(2n+1) Y_n^m and the interior one
    n/(2n+1) Y_n^m (S[Y_n^m] = r^n Y_n^m/(2n+1) inside, r^-(n+1) Y_n^m/(2n+1) outside).  Sources from a 4x
    finer mesh than the centers, as in the potential's closed-form pin."""
    from paper_1805_06106_gb300.solve import normal_derivative, normal_derivative_targets
    from synth import make_surface, real_ylm

    sc, ss = make_surface(2), make_surface(8)
    sub = np.random.default_rng(0).choice(sc.n_src, 40, replace=False)
    k = sub.size
    sig = real_ylm(n, m, ss.src_xyz)
    Y = real_ylm(n, m, sc.src_xyz[:, sub])
    for offset, limit in ((0, -(n + 1) / (2 * n + 1)), (sc.n_src, n / (2 * n + 1))):
        h = 1e-2 * sc.ctr_r[sub]
        tp = normal_derivative_targets(sc.src_xyz[:, sub], sc.src_n[:, sub], h)
        ctr = np.concatenate([sc.ctr_xyz[:, sub + offset]] * 2, axis=1)
        pot = O.direct_eval(ss.src_xyz, ss.src_w, sig, None, ss.src_n, ctr, tp, np.arange(2 * k, dtype=np.int32), 7)
        d = normal_derivative(pot, h)
        assert np.max(np.abs(d - limit * Y)) / np.max(np.abs(limit * Y)) < 1e-2
