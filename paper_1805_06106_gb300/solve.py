"""Boundary-value problems solved with the evaluation as the operator (the use of Section 6.2), and the
normal derivative S' of the single layer at targets from the same evaluation.

The QBX evaluation gives one-sided limits of layer potentials on the surface: a target evaluated
through its interior center receives the interior limit.  For the interior Dirichlet problem of the
Laplace equation the solution is sought as a double-layer potential u = D[mu]; on the surface its
interior limit is the second-kind operator D^-[mu] = -mu/2 + K[mu], and D^-[mu] = f is solved for mu by
restarted GMRES.  The density is a polynomial of degree 4 per element given by its values at 15
interior collocation nodes; the sources are the nodes of an oversampled (stage-2) rule and receive
the density through the element's interpolation matrix, so that the QBX coefficients are integrated
accurately (Section 3.3).  Each operator application is one GIGAQBX evaluation (qbx_eval).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding as B


def gmres(matvec, b, tol=1e-10, restart=40, maxiter=400):
    """Restarted GMRES (Arnoldi with modified Gram-Schmidt, Givens rotations) for A x = b.  matvec maps
    a tensor like b to A times it.  Stops when the residual estimate reaches tol |b|.  Returns
    (x, info), info = {"iterations", "converged", "residuals" (relative, per iteration; the last entry
    the true residual of the returned x)}."""
    x = torch.zeros_like(b)
    bnorm = float(torch.linalg.vector_norm(b))
    if bnorm == 0.0:
        return x, {"iterations": 0, "converged": True, "residuals": [0.0]}
    hist, total, converged = [], 0, False
    while total < maxiter and not converged:
        r = b - matvec(x)
        beta = float(torch.linalg.vector_norm(r))
        if beta <= tol * bnorm:
            converged = True
            break
        m = min(restart, maxiter - total)
        V = [r / beta]
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        for j in range(m):
            w = matvec(V[j])
            total += 1
            for i in range(j + 1):
                H[i, j] = float(torch.dot(w, V[i]))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(torch.linalg.vector_norm(w))
            breakdown = H[j + 1, j] <= 1e-300
            if not breakdown:
                V.append(w / H[j + 1, j])
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j], H[j + 1, j] = d, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or breakdown:
                converged = True
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):  # back substitution with the triangular H[:k, :k]
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        for i in range(k):
            x = x + float(y[i]) * V[i]
    hist.append(float(torch.linalg.vector_norm(b - matvec(x))) / bnorm)
    return x, {"iterations": total, "converged": converged, "residuals": hist}


def interpolate(interp, mu_nodes):
    """Density at the sources from its values at the collocation nodes, element by element
    (interp: (sources, nodes) per element, a tensor on mu_nodes' device)."""
    n_nodes = interp.shape[1]
    return (mu_nodes.reshape(-1, n_nodes) @ interp.T).reshape(-1)


def dirichlet_double_layer(apply_interior_dlp, interp, f, tol=1e-10, restart=60, maxiter=600):
    """Density mu (at the collocation nodes) with D^-[mu] = f.  apply_interior_dlp(mu_src) returns the
    interior limit of D[mu_src] at the collocation nodes for a density given at the sources."""
    return gmres(lambda mu: apply_interior_dlp(interpolate(interp, mu)), f, tol=tol, restart=restart,
                 maxiter=maxiter)


def interior_dirichlet(tree, lists, src_w, src_n, tgt_ctr, interp, f, p_qbx, p_fmm, precision=B.QBX_FP64,
                       tol=1e-10, restart=60, maxiter=600):
    """dirichlet_double_layer with qbx_eval as the operator: `tree`'s targets are the collocation nodes,
    each associated through tgt_ctr with its interior center; its sources carry src_w and src_n (device
    arrays).  Returns (mu at the nodes, GMRES info)."""
    out = torch.empty_like(f)

    def apply(mu_src):
        B.qbx_eval(tree, lists, src_w, None, mu_src, src_n, tgt_ctr, p_qbx, p_fmm, precision=precision, out=out)
        return out.clone()

    return dirichlet_double_layer(apply, interp, f, tol=tol, restart=restart, maxiter=maxiter)


def normal_derivative_targets(tgt_xyz, tgt_n, h):
    """Targets for S' (the normal derivative at the targets of the single layer, Section 2): the points
    t + h n_t (first half) and t - h n_t (second half), (3, 2 N_T); evaluate both halves through the
    centers of the targets t (tgt_ctr repeated twice) and pass the result to normal_derivative."""
    t, n = np.asarray(tgt_xyz), np.asarray(tgt_n)
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (t.shape[1],))
    return np.concatenate([t + h * n, t - h * n], axis=1)


def normal_derivative(pot_pm, h):
    """S'[sigma] = d/dn_t S[sigma] at each target from the potentials at t +- h n_t: the central difference
    of the target's QBX local expansion (a polynomial in t - c, the same expansion for both points, so
    the limit from the center's side is kept and the error is O(h^2) plus rounding / h; h about 1e-2
    of the expansion radius)."""
    n = pot_pm.shape[0] // 2
    return (pot_pm[:n] - pot_pm[n:]) / (2.0 * h)


def single_layer_normal_derivative(tree, lists, src_w, sigma, src_n, tgt_ctr_pm, h, p_qbx, p_fmm,
                                   precision=B.QBX_FP64):
    """S'[sigma] at N_T targets on the GPU: `tree` built with normal_derivative_targets' points as its
    targets, tgt_ctr_pm the targets' centers twice (device int32, 2 N_T), h the step per target
    (a device tensor or a number).  One qbx_eval, then normal_derivative."""
    pot = B.qbx_eval(tree, lists, src_w, sigma, None, src_n, tgt_ctr_pm, p_qbx, p_fmm, precision=precision)
    return normal_derivative(pot, h)
