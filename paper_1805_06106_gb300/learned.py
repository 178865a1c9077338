"""Learned expansion orders: order sweeps -> labels -> MLP training -> per-center / per-box orders,
checked against the fixed-order evaluation (the judge) with a fallback.

Host-side orchestration only; every arithmetic step (features, labels, network forward, backward
and Adam, order assignment, judge and fallback, evaluations) runs in libqbx kernels.

Labels (per center, relative to the fixed orders (q_fix, p_fix) of the judge):
  p_qbx label = lowest q <= q_fix whose truncated QBX local stays within label_frac * tol (normwise,
  relative to max |phi|) of the order-q_fix result for every order from q up (one order sweep);
  p_fmm label = lowest p of the grid such that the evaluation with every box's local expansion of
  order p (multipoles keep p_fix) stays within label_frac * tol of the fixed-order result for every
  grid order from p up.  A box's order is the largest prediction over the centers below it.
Per-box orders compose truncations that a uniform sweep does not see (a box at order p below a parent
of higher order), so some centers miss the tolerance their labels promise.  The judge finds them: one
fixed-order evaluation of the problem, and every target that misses raises its center's QBX order and
its box chain's local orders to the fixed orders (qbx_orders_fallback), until none misses.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import binding as B

P_GRID = (4, 5, 6, 7, 8, 9, 10, 11, 12, 14, 16, 18, 20)


@dataclass
class Samples:
    x: torch.Tensor  # (n, 4) float32 features
    y: torch.Tensor  # (n, 2) float32 labels (p_qbx, p_fmm)


@dataclass
class Model:
    params: torch.Tensor           # QBX_MLP_NPARAMS float32 on the device
    margin_q: float                # added to the predicted QBX order before rounding up
    margin_p: float                # added to the predicted local order before rounding up
    losses: list = field(default_factory=list)


def _cu(a, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()


def sweep_samples(surf, sigma, mu, q_fix, p_fix, n_max, tol, label_frac=0.25, precision=B.QBX_FP64):
    """Features and labels of every center of one surface whose targets are one on-surface target
    per center, in center order (tgt_ctr[t] = t)."""
    if not np.array_equal(np.asarray(surf.tgt_ctr), np.arange(surf.n_ctr)):
        raise ValueError("training surfaces carry one on-surface target per center, in center order")
    T = B.qbx_build_tree(_cu(surf.src_xyz), _cu(surf.ctr_xyz), _cu(surf.ctr_r), _cu(surf.tgt_xyz), n_max=n_max)
    L = B.qbx_build_lists(T)
    args = (_cu(surf.src_w), None if sigma is None else _cu(sigma), None if mu is None else _cu(mu),
            _cu(surf.src_n), _cu(surf.tgt_ctr, torch.int32))
    feats = B.qbx_center_features(T, L, args[0], args[1], args[2], args[3])
    part = B.qbx_eval_order_sweep(T, L, *args, q_fix, p_fix, precision=precision)
    scale = float(part[q_fix].abs().max())
    qlab = B.qbx_order_labels(part[: q_fix + 1], list(range(q_fix + 1)), label_frac * tol * scale)
    grid = [p for p in P_GRID if p < p_fix] + [p_fix]
    vals = []
    for p in grid:
        pb = torch.full((T.n_boxes,), p, dtype=torch.int8, device="cuda")
        vals.append(B.qbx_eval(T, L, *args, q_fix, p_fix, p_fmm_per_box=pb, precision=precision))
    plab = B.qbx_order_labels(torch.stack(vals), grid, label_frac * tol * scale)
    return Samples(feats, torch.stack([qlab.float(), plab.float()], dim=1))


def fit(samples, steps=1500, lr=3e-3, seed=0, chunk=250, quantile=0.9):
    """Full-batch Adam on the concatenated samples with the library's kernels, then margins: the
    given quantile of (label - prediction) over the training samples, plus half an order."""
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
    res = y.cpu().numpy() - B.qbx_mlp_forward(params, x).cpu().numpy()
    mq, mp = (float(max(0.0, np.quantile(res[:, k], quantile)) + 0.5) for k in range(2))
    return Model(params, mq, mp, losses)


def predict_orders(tree, lists, model, src_w, sigma, mu, src_n, tgt_ctr=None, q_range=(2, 12), p_range=(4, 20),
                   p_default=16):
    """Per-center QBX orders and per-box local-expansion orders of one problem (tgt_ctr marks point
    targets, whose boxes keep the highest order)."""
    feats = B.qbx_center_features(tree, lists, src_w, sigma, mu, src_n)
    pred = B.qbx_mlp_forward(model.params, feats)
    return B.qbx_orders_from_mlp(tree, lists, pred, model.margin_q, model.margin_p, q_range[0], q_range[1],
                                 p_range[0], p_range[1], p_default, tgt_ctr=tgt_ctr)


def judge_and_fallback(tree, lists, args, q_fix, p_fix, qc, pb, tol, precision, judge=None, max_rounds=4):
    """Evaluate with the learned orders, compare with the fixed-order FP64 judge and raise the orders
    where a target misses tol * scale; repeat until no target misses.  scale = max|judge| over the
    problem, or for a forest the smallest such maximum over its problems (so that every problem meets
    tol in its own normwise measure).  args = (src_w, sigma, mu, src_n, tgt_ctr).  Returns (qc, pb,
    info); qc and pb are updated in place; info["err_before"] / ["err_after"] are max|res - judge| /
    scale before and after."""
    if judge is None:
        judge = B.qbx_eval(tree, lists, *args, q_fix, p_fix)
    off = getattr(tree, "offsets", None)
    if off is not None:
        t = off["tgt"]
        scale = min(float(judge[t[i]:t[i + 1]].abs().max()) for i in range(len(t) - 1) if t[i + 1] > t[i])
    else:
        scale = float(judge.abs().max())
    thr = tol * scale
    info = {"rounds": 0, "raised": [], "err_before": None, "err_after": None}
    for r in range(max_rounds + 1):
        res = B.qbx_eval(tree, lists, *args, q_fix, p_fix, p_qbx_per_ctr=qc, p_fmm_per_box=pb, precision=precision)
        err = float((res - judge).abs().max()) / scale
        if r == 0:
            info["err_before"] = err
        info["err_after"] = err
        if r == max_rounds:
            break
        n = B.qbx_orders_fallback(tree, res, judge, args[4], thr, q_fix, p_fix, qc, pb)
        info["raised"].append(n)
        if n == 0:
            break
        info["rounds"] = r + 1
    return qc, pb, info


def save(model, path):
    np.savez(path, params=model.params.detach().cpu().numpy(), margins=np.array([model.margin_q, model.margin_p]))


def load(path):
    d = np.load(path)
    return Model(torch.from_numpy(d["params"]).cuda(), float(d["margins"][0]), float(d["margins"][1]))
