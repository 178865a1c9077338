"""Learned expansion orders: order sweeps -> labels -> MLP training -> per-center / per-box orders.

Host-side orchestration only; every arithmetic step (features, labels, network forward,
backward and Adam, order assignment, evaluations) runs in libqbx kernels.

Labels (per center, relative to the fixed orders (q_fix, p_fix) that act as the acceptance check):
  p_qbx label = lowest q <= q_fix whose truncated QBX local stays within tol/2 (normwise, relative
  to max |phi|) of the order-q_fix result for every order from q to q_fix (one order sweep);
  p_fmm label = lowest p in the grid whose result at (q_fix, p) stays within tol/2 of the
  (q_fix, p_fix) result for every grid order from p to p_fix.
A center's associated target supplies its labels (one on-surface target per center).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import binding as B

P_GRID = (4, 6, 8, 10, 12, 14, 16, 18, 20)


@dataclass
class Samples:
    x: torch.Tensor  # (n, 4) float32 features
    y: torch.Tensor  # (n, 2) float32 labels (p_qbx, p_fmm)


def sweep_samples(surf, sigma, mu, q_fix, p_fix, n_max, tol, precision=B.QBX_M2L_FP32):
    """Features and labels of every center of one surface (targets = one per center)."""
    cu = lambda a, dt=torch.float64: torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()  # noqa: E731
    T = B.qbx_build_tree(cu(surf.src_xyz), cu(surf.ctr_xyz), cu(surf.ctr_r), cu(surf.tgt_xyz), n_max=n_max)
    L = B.qbx_build_lists(T)
    args = (cu(surf.src_w), None if sigma is None else cu(sigma), None if mu is None else cu(mu), cu(surf.src_n),
            cu(surf.tgt_ctr, torch.int32))
    feats = B.qbx_center_features(T, L, args[0], args[1], args[2], args[3])
    part = B.qbx_eval_order_sweep(T, L, *args, q_fix, p_fix, precision=precision)
    scale = float(part[q_fix].abs().max())
    qlab = B.qbx_order_labels(part[: q_fix + 1], list(range(q_fix + 1)), 0.5 * tol * scale)
    grid = [p for p in P_GRID if q_fix <= p <= p_fix]
    if grid[-1] != p_fix:
        grid.append(p_fix)
    vals = torch.stack([B.qbx_eval(T, L, *args, q_fix, p, precision=precision) for p in grid])
    plab = B.qbx_order_labels(vals, grid, 0.5 * tol * scale)
    y = torch.stack([qlab.float(), plab.float()], dim=1)
    return Samples(feats, y)


def train(samples, steps=1500, lr=3e-3, seed=0, chunk=250):
    """Full-batch Adam on the concatenated samples with the library's kernels."""
    x = torch.cat([s.x for s in samples]).contiguous()
    y = torch.cat([s.y for s in samples]).contiguous()
    params = B.qbx_mlp_init(seed)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    losses = []
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        losses.append(B.qbx_mlp_train(params, m, v, x, y, k, done + 1, lr))
        done += k
    return params, losses


def calibrate(params, samples, quantile=0.999):
    """Margins that make ceil(prediction + margin) cover the training labels: the given quantile of
    (label - prediction) over the training samples, plus half an order."""
    x = torch.cat([s.x for s in samples]).contiguous()
    y = torch.cat([s.y for s in samples]).cpu().numpy()
    pred = B.qbx_mlp_forward(params, x).cpu().numpy()
    res = y - pred
    return tuple(float(max(0.0, np.quantile(res[:, k], quantile)) + 0.5) for k in range(2))


def predict_orders(tree, lists, params, src_w, sigma, mu, src_n, q_range=(2, 12), p_range=(4, 20),
                   margin_q=0.5, margin_p=1.0, p_default=16, tgt_ctr=None):
    """Per-center QBX orders and per-box local-expansion orders for one surface (tgt_ctr marks its
    point targets, whose boxes keep the highest order)."""
    feats = B.qbx_center_features(tree, lists, src_w, sigma, mu, src_n)
    pred = B.qbx_mlp_forward(params, feats)
    return B.qbx_orders_from_mlp(tree, lists, pred, margin_q, margin_p, q_range[0], q_range[1], p_range[0],
                                 p_range[1], p_default, tgt_ctr=tgt_ctr)


def save(params, path):
    np.save(path, params.detach().cpu().numpy())


def load(path):
    return torch.from_numpy(np.load(path)).cuda()
