"""Quadrature rules on the triangle built by node elimination (the construction of Xiao and Gimbutas,
2010, that the paper's stage-2 quadrature uses, Section 3.1): start from a conical-product rule exact
to total degree d, then repeatedly drop the least significant node and restore exactness by
Gauss-Newton on the moment equations (nodes and weights free, least-norm steps), keeping a removal
only when the new rule is exact to rounding with every node inside the triangle and every weight
positive.  The rules here are not forced to be symmetric (the published rules are); they serve as
the oversampled source quadrature of the stage-2 discretization.

The moment equations are written in an orthogonal (Dubiner / Koornwinder) basis of the polynomials
of degree <= d on the unit triangle {u, v >= 0, u + v <= 1}: psi_pq = L_p(u, v) P_q^(2p+1, 0)(2v - 1),
L_p the Legendre polynomial of (2u + v - 1) / (1 - v) times (1 - v)^p, evaluated by its homogeneous
three-term recurrence so that it stays a polynomial up to the vertex v = 1.
"""
from __future__ import annotations

import functools
import math

import numpy as np
import torch


def _basis(u, v, d):
    """(M, N) values of psi_pq, p + q <= d, at points (u, v) (torch, float64)."""
    x, t = 2.0 * u + v - 1.0, 1.0 - v
    L = [torch.ones_like(u), x]
    for n in range(1, d):
        L.append(((2 * n + 1) * x * L[n] - n * t * t * L[n - 1]) / (n + 1))
    b = 2.0 * v - 1.0
    out = []
    for p in range(d + 1):
        a = 2 * p + 1
        P = [torch.ones_like(u), 0.5 * ((a + 2) * b + a)]  # Jacobi P^(a, 0)
        for n in range(2, d - p + 1):
            c0 = 2 * n * (n + a) * (2 * n + a - 2)
            c1 = (2 * n + a - 1) * ((2 * n + a) * (2 * n + a - 2) * b + a * a)
            c2 = 2 * (n + a - 1) * (n - 1) * (2 * n + a)
            P.append((c1 * P[n - 1] - c2 * P[n - 2]) / c0)
        for q in range(d - p + 1):
            out.append(L[p] * P[q])
    return torch.stack(out)


def _norms(d):
    """Integrals of psi_pq^2 over the triangle (a conical rule exact to degree 2d)."""
    u, v, w = (torch.from_numpy(a) for a in _conical(d + 1))
    B = _basis(u, v, d)
    return (B * B * w).sum(dim=1)


def _conical(n):
    from .surfaces import conical_rule

    return conical_rule(n)


def _gauss_newton(u, v, w, d, scale, iters=40):
    """Moment equations sum_i w_i psi_j(x_i) = int psi_j (only psi_00 = 1 has a nonzero integral, 1/2),
    rows scaled to unit norm.  Returns (u, v, w, residual) after least-norm Gauss-Newton steps."""
    target = torch.zeros(scale.shape[0], dtype=torch.float64)
    target[0] = 0.5
    z = torch.cat([u, v, w]).clone()
    n = u.shape[0]

    def F(z):
        return (_basis(z[:n], z[n:2 * n], d) @ z[2 * n:] - target) / scale

    r = F(z)
    for _ in range(iters):
        if float(r.abs().max()) < 1e-15:
            break
        J = torch.autograd.functional.jacobian(F, z, vectorize=True)
        step = torch.linalg.lstsq(J, -r.unsqueeze(1), driver="gelsd").solution.squeeze(1)
        z = z + step
        r = F(z)
    return z[:n], z[n:2 * n], z[2 * n:], float(r.abs().max())


def _valid(u, v, w):
    return bool((u > 0).all() and (v > 0).all() and (u + v < 1).all() and (w > 0).all())


@functools.lru_cache(maxsize=None)
def eliminated_rule(d: int, max_tries: int = 12):
    """A rule exact to total degree d on the unit triangle with fewer nodes than the conical-product
    rule it starts from.  Returns (u, v, w) numpy arrays (sum(w) = 1/2)."""
    n0 = (d + 2) // 2  # conical rule with n0^2 nodes is exact to 2 n0 - 1 >= d
    u, v, w = (torch.from_numpy(a.copy()) for a in _conical(n0))
    scale = torch.sqrt(_norms(d))
    while True:
        B = _basis(u, v, d) / scale[:, None]
        significance = w * (B * B).sum(dim=0)
        done = True
        for i in torch.argsort(significance).tolist()[:max_tries]:
            keep = torch.ones(u.shape[0], dtype=torch.bool)
            keep[i] = False
            nu, nv, nw, res = _gauss_newton(u[keep], v[keep], w[keep], d, scale)
            if res < 1e-14 and _valid(nu, nv, nw):
                u, v, w = nu, nv, nw
                done = False
                break
        if done:
            return u.numpy(), v.numpy(), w.numpy()


def exactness_error(u, v, w, d):
    """Largest error of the rule on the monomials u^a v^b, a + b <= d (exact value a! b! / (a + b + 2)!)."""
    return max(abs(float(np.sum(w * u ** a * v ** b)) - math.factorial(a) * math.factorial(b) /
                   math.factorial(a + b + 2)) for a in range(d + 1) for b in range(d + 1 - a))
