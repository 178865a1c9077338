"""ctypes front end of the FP64 CPU oracle (oracle/qbx_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py.  The product library never loads it.

Coefficient arrays are complex128 of length (p+1)^2, ordered
B_0^0, B_1^-1, B_1^0, B_1^1, ... (Section 4.1).  Point arrays are SoA (3, N)
float64.  Lists are CSR (start[n_boxes+1], idx) in the order
U, V, W-close, W-far, X-close, X-far (Section 5.2.3-5.2.4).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qbx_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")
_LIB_OMP = os.path.join(_HERE, "_build", "liborc_omp.so")  # the same source built with -fopenmp

LIST_NAMES = ("U", "V", "Wclose", "Wfar", "Xclose", "Xfar")


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2 -ffp-contract=off, no target-specific flags): a serial library
    and, where the compiler supports it, the same source with OpenMP (all-cores timing only)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    base = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared"]
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.run(base + ["-o", _LIB, _SRC, "-lm"], check=True)
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        subprocess.run(base + ["-fopenmp", "-o", _LIB_OMP, _SRC, "-lm"], check=False)
    return _LIB


_lib = None
_lib_omp = None


def lib_omp():
    """The OpenMP build (same functions; orc_fmm_eval runs its box and center loops on all cores)."""
    global _lib_omp
    if _lib_omp is None:
        lib()
        if not os.path.exists(_LIB_OMP):
            raise RuntimeError("the OpenMP build of the oracle is not available (gcc -fopenmp failed)")
        L = C.CDLL(_LIB_OMP)
        P = C.c_void_p
        i = C.c_int
        L.orc_fmm_eval.argtypes = [P, P, P, i, P, P, P, P, P, i, P, P, i, i, i, P, P, P, P, i]
        _lib_omp = L
    return _lib_omp


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        d, i = C.c_double, C.c_int
        L.orc_ylm.argtypes = [i, P, P]
        L.orc_p2m.argtypes = [i, P, P, d, P, P]
        L.orc_p2l.argtypes = [i, P, P, d, P, P]
        L.orc_m2p.argtypes = [i, P, P, P]
        L.orc_m2p.restype = d
        L.orc_l2p.argtypes = [i, P, P, P]
        L.orc_l2p.restype = d
        L.orc_p2p.argtypes = [P, d, P, P]
        L.orc_p2p.restype = d
        for f in (L.orc_m2m, L.orc_l2l, L.orc_m2l):
            f.argtypes = [i, P, P, i, P, P]
        L.orc_build_tree.argtypes = [P, i, P, P, i, P, i, i, d, i, i]
        L.orc_build_tree.restype = P
        L.orc_tree_free.argtypes = [P]
        L.orc_tree_info.argtypes = [P, P, P]
        L.orc_tree_arrays.argtypes = [P] * 10
        for f in (L.orc_build_lists, L.orc_build_lists_slow):
            f.argtypes = [P]
            f.restype = P
        L.orc_lists_free.argtypes = [P]
        L.orc_lists_nnz.argtypes = [P, i]
        L.orc_lists_nnz.restype = C.c_int64
        L.orc_lists_get.argtypes = [P, i, P, P]
        L.orc_fmm_eval.argtypes = [P, P, P, i, P, P, P, P, P, i, P, P, i, i, i, P, P, P, P, i]
        L.orc_direct_eval.argtypes = [P, i, P, P, P, P, P, i, P, P, i, i, P, P]
        L.orc_lists_cost.argtypes = [P, P, i, i, P]
        L.orc_lists_counts.argtypes = [P, P, P]
        L.orc_mlp_loss_grad.argtypes = [P, P, P, i, P]
        L.orc_mlp_loss_grad_f64.argtypes = [P, P, P, i, P]
        L.orc_order_labels.argtypes = [P, i, P, i, d, P]
        L.orc_orders_from_pred.argtypes = [P, P, P, C.c_float, C.c_float, i, i, i, i, i, P, P]
        L.orc_center_features.argtypes = [P, P, P, P, P, P, P, P, P]
        L.orc_orders_fallback.argtypes = [P, P, P, P, d, i, i, P, P]
        L.orc_assoc_targets.argtypes = [P, P, P, P, P, P, P, P, d, P, P]
        L.orc_refine_marks.argtypes = [i, P, i, P, P, i, P, P, i, d, P]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _ncoef(p):
    return (p + 1) * (p + 1)


# ---------------------------------------------------------------- operators


def ylm(p, v):
    out = np.zeros(_ncoef(p), np.complex128)
    v = _f64(v)
    if lib().orc_ylm(p, _p(v), _p(out)) != 0:
        raise ValueError("ylm of the zero vector")
    return out


def p2m(p, c, s, q, d=None):
    out = np.zeros(_ncoef(p), np.complex128)
    c, s, d = _f64(c), _f64(s), _f64(d)
    lib().orc_p2m(p, _p(c), _p(s), float(q), _p(d), _p(out))
    return out


def p2l(p, c, s, q, d=None):
    out = np.zeros(_ncoef(p), np.complex128)
    c, s, d = _f64(c), _f64(s), _f64(d)
    lib().orc_p2l(p, _p(c), _p(s), float(q), _p(d), _p(out))
    return out


def m2p(p, c, M, t):
    c, t, M = _f64(c), _f64(t), np.ascontiguousarray(M, np.complex128)
    return lib().orc_m2p(p, _p(c), _p(M), _p(t))


def l2p(p, c, L, t):
    c, t, L = _f64(c), _f64(t), np.ascontiguousarray(L, np.complex128)
    return lib().orc_l2p(p, _p(c), _p(L), _p(t))


def p2p(s, q, t, d=None):
    s, t, d = _f64(s), _f64(t), _f64(d)
    return lib().orc_p2p(_p(s), float(q), _p(d), _p(t))


def _translate(fn, ps, c, B, pd, c2):
    out = np.zeros(_ncoef(pd), np.complex128)
    c, c2, B = _f64(c), _f64(c2), np.ascontiguousarray(B, np.complex128)
    fn(ps, _p(c), _p(B), pd, _p(c2), _p(out))
    return out


def m2m(ps, c, M, pd, c2):
    return _translate(lib().orc_m2m, ps, c, M, pd, c2)


def l2l(ps, c, L, pd, c2):
    return _translate(lib().orc_l2l, ps, c, L, pd, c2)


def m2l(ps, c, M, pd, c2):
    return _translate(lib().orc_m2l, ps, c, M, pd, c2)


# ---------------------------------------------------------------- tree and lists


@dataclass
class Tree:
    handle: int
    n_boxes: int
    n_levels: int
    n_overfull: int
    root_center: np.ndarray
    root_radius: float
    level: np.ndarray
    coords: np.ndarray  # (n_boxes, 3) int64
    center: np.ndarray  # (n_boxes, 3)
    radius: np.ndarray  # |b|
    parent: np.ndarray
    child: np.ndarray  # (n_boxes, 8)
    src_owner: np.ndarray
    ctr_owner: np.ndarray
    tgt_owner: np.ndarray

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.orc_tree_free(self.handle)
            self.handle = 0


def build_tree(src_xyz, ctr_xyz, ctr_r, tgt_xyz, n_max=32, t_f=0.9, max_depth=40, linf_tcr=False,
               level_restrict=False) -> Tree:
    """Stage 1 tree.  linf_tcr: the box-shaped (l-infinity) TCR of Table l2-comparison's left
    columns; level_restrict: adjacent leaves differ by at most one level (Remark on level
    restriction, Section 5.3)."""
    s, c, r, t = _f64(src_xyz), _f64(ctr_xyz), _f64(ctr_r), _f64(tgt_xyz)
    ns, nc, nt = s.shape[1], c.shape[1], t.shape[1]
    flags = (1 if linf_tcr else 0) | (2 if level_restrict else 0)
    h = lib().orc_build_tree(_p(s), ns, _p(c), _p(r), nc, _p(t), nt, n_max, t_f, max_depth, flags)
    info = np.zeros(6, np.int64)
    root = np.zeros(4)
    lib().orc_tree_info(h, _p(info), _p(root))
    nb = int(info[0])
    arr = dict(level=np.zeros(nb, np.int32), coords=np.zeros((nb, 3), np.int64), center=np.zeros((nb, 3)),
               radius=np.zeros(nb), parent=np.zeros(nb, np.int32), child=np.zeros((nb, 8), np.int32),
               src_owner=np.zeros(ns, np.int32), ctr_owner=np.zeros(nc, np.int32), tgt_owner=np.zeros(nt, np.int32))
    lib().orc_tree_arrays(h, *[_p(arr[k]) for k in ("level", "coords", "center", "radius", "parent", "child",
                                                        "src_owner", "ctr_owner", "tgt_owner")])
    return Tree(h, nb, int(info[1]), int(info[2]), root[:3].copy(), float(root[3]), **arr)


@dataclass
class Lists:
    handle: int
    start: dict
    idx: dict

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.orc_lists_free(self.handle)
            self.handle = 0

    def of(self, name, b):
        return self.idx[name][self.start[name][b]:self.start[name][b + 1]]


def build_lists(tree: Tree, slow: bool = False) -> Lists:
    h = (lib().orc_build_lists_slow if slow else lib().orc_build_lists)(tree.handle)
    start, idx = {}, {}
    for k, name in enumerate(LIST_NAMES):
        nnz = lib().orc_lists_nnz(h, k)
        st = np.zeros(tree.n_boxes + 1, np.int32)
        ix = np.zeros(max(nnz, 1), np.int32)
        lib().orc_lists_get(h, k, _p(st), _p(ix))
        start[name], idx[name] = st, ix[:nnz]
    return Lists(h, start, idx)


def lists_counts(tree: Tree, lists: Lists) -> dict:
    """Interaction counts per list: sum of n_s n_t (U, W-close, X-close), entries (V), sum of n_t
    (W-far), sum of subtree n_s (X-far); n_t = QBX centers of the target box."""
    out = np.zeros(6, np.int64)
    lib().orc_lists_counts(tree.handle, lists.handle, _p(out))
    return dict(zip(LIST_NAMES, (int(v) for v in out)))


def lists_cost(tree: Tree, lists: Lists, p_qbx: int, p_fmm: int) -> dict:
    """Modeled operation counts: per list (Table ilist-operation-counts), the remaining stage
    terms of Table complexity-analysis ("stages"), and their sum ("total")."""
    out = np.zeros(8)
    lib().orc_lists_cost(tree.handle, lists.handle, p_qbx, p_fmm, _p(out))
    return dict(zip(LIST_NAMES + ("stages", "total"), out.tolist()))


# ---------------------------------------------------------------- evaluation


def fmm_eval(tree: Tree, lists: Lists, src_xyz, src_w, sigma, mu, src_n, ctr_xyz, tgt_xyz, tgt_ctr,
             p_qbx, p_fmm, p_qbx_ctr=None, p_fmm_box=None, return_qbx_locals=False, qmax=None, omp=False):
    """GIGAQBX FMM (Algorithm 4): pot = S[sigma] + D[mu] at every target.  omp=True runs the OpenMP
    build of the same code (same results)."""
    s, w, sg, m_, n_ = _f64(src_xyz), _f64(src_w), _f64(sigma), _f64(mu), _f64(src_n)
    c, t = _f64(ctr_xyz), _f64(tgt_xyz)
    tc = np.ascontiguousarray(tgt_ctr, np.int32)
    qc = None if p_qbx_ctr is None else np.ascontiguousarray(p_qbx_ctr, np.int8)
    pb = None if p_fmm_box is None else np.ascontiguousarray(p_fmm_box, np.int8)
    nt = t.shape[1]
    pot = np.zeros(nt)
    qm = qmax if qmax is not None else (p_qbx if qc is None else int(qc.max()))
    ql = np.zeros((c.shape[1], _ncoef(qm)), np.complex128) if return_qbx_locals else None
    rc = (lib_omp() if omp else lib()).orc_fmm_eval(tree.handle, lists.handle, _p(s), s.shape[1], _p(w), _p(sg), _p(m_), _p(n_), _p(c),
                            c.shape[1], _p(t), _p(tc), nt, p_qbx, p_fmm, _p(qc), _p(pb), _p(pot), _p(ql), qm)
    if rc != 0:
        raise ValueError("particle counts do not match the tree")
    return (pot, ql) if return_qbx_locals else pot


def direct_eval(src_xyz, src_w, sigma, mu, src_n, ctr_xyz, tgt_xyz, tgt_ctr, p_qbx, p_qbx_ctr=None):
    """Direct (unaccelerated) QBX, eqs. (qbxcoeff) and (qbxlocal); point targets by plain quadrature."""
    s, w, sg, m_, n_ = _f64(src_xyz), _f64(src_w), _f64(sigma), _f64(mu), _f64(src_n)
    c, t = _f64(ctr_xyz), _f64(tgt_xyz)
    tc = np.ascontiguousarray(tgt_ctr, np.int32)
    qc = None if p_qbx_ctr is None else np.ascontiguousarray(p_qbx_ctr, np.int8)
    pot = np.zeros(t.shape[1])
    lib().orc_direct_eval(_p(s), s.shape[1], _p(w), _p(sg), _p(m_), _p(n_), _p(c), c.shape[1], _p(t), _p(tc),
                          t.shape[1], p_qbx, _p(qc), _p(pot))
    return pot


# ---------------------------------------------------------------- learned-order network


def mlp_loss_grad(params, x, target):
    """Gradient (4610 values) and loss of the 4-64-64-2 tanh network, FP64 chain rule."""
    p = np.ascontiguousarray(params, np.float32)
    xx = np.ascontiguousarray(x, np.float32)
    tt = np.ascontiguousarray(target, np.float32)
    out = np.zeros(p.size + 1)
    lib().orc_mlp_loss_grad(_p(p), _p(xx), _p(tt), xx.shape[0], _p(out))
    return out[:-1], out[-1]


def mlp_loss_grad_f64(params, x, target):
    """The same gradient and loss with double-precision parameters, inputs and labels."""
    p = np.ascontiguousarray(params, np.float64)
    xx = np.ascontiguousarray(x, np.float64)
    tt = np.ascontiguousarray(target, np.float64)
    out = np.zeros(p.size + 1)
    lib().orc_mlp_loss_grad_f64(_p(p), _p(xx), _p(tt), xx.shape[0], _p(out))
    return out[:-1], out[-1]


def center_features(tree: Tree, lists: Lists, src_w, sigma, mu, src_n, ctr_xyz, ctr_r):
    """(n_ctr, 4) float32 inputs of the order network per center (input order)."""
    w, sg, m_, n_ = _f64(src_w), _f64(sigma), _f64(mu), _f64(src_n)
    c, r = _f64(ctr_xyz), _f64(ctr_r)
    out = np.zeros((c.shape[1], 4), np.float32)
    lib().orc_center_features(tree.handle, lists.handle, _p(w), _p(sg), _p(m_), _p(n_), _p(c), _p(r), _p(out))
    return out


def orders_fallback(tree: Tree, res, judge, tgt_ctr, tol, q_fix, p_fix, q, pb):
    """Raise in place the orders of centers and box chains whose targets miss the judge; returns the
    number of such targets.  q (n_ctr,) and pb (n_boxes,) are int32 arrays."""
    r, j = _f64(res), _f64(judge)
    tc = np.ascontiguousarray(tgt_ctr, np.int32)
    assert q.dtype == np.int32 and pb.dtype == np.int32 and q.flags.c_contiguous and pb.flags.c_contiguous
    return int(lib().orc_orders_fallback(tree.handle, _p(r), _p(j), _p(tc), float(tol), q_fix, p_fix, _p(q), _p(pb)))


def assoc_targets(tree: Tree, src_xyz, rdanger, src_n, ctr_xyz, ctr_r, ctr_side, tgt_xyz, eps):
    """Target association (Algorithm 3 with the area queries of Algorithm 5): (tgt_ctr int32 with -1
    for none, flagged bool) per target of the tree.  src_n / ctr_side None: no side preference."""
    sx, rd, c, r, t = _f64(src_xyz), _f64(rdanger), _f64(ctr_xyz), _f64(ctr_r), _f64(tgt_xyz)
    sn = None if src_n is None else _f64(src_n)
    cs = None if ctr_side is None else np.ascontiguousarray(ctr_side, np.int8)
    nt = t.shape[1]
    tc = np.zeros(nt, np.int32)
    fl = np.zeros(nt, np.int32)
    lib().orc_assoc_targets(tree.handle, _p(sx), _p(rd), _p(sn), _p(c), _p(r), _p(cs), _p(t), float(eps), _p(tc),
                            _p(fl))
    return tc, fl.astype(bool)


def order_labels(values, orders, tol):
    """values (K, n) results at increasing orders (last = reference) -> (n,) labels."""
    v = np.ascontiguousarray(values, np.float64)
    o = np.ascontiguousarray(orders, np.int32)
    out = np.zeros(v.shape[1], np.int32)
    lib().orc_order_labels(_p(v), v.shape[0], _p(o), v.shape[1], float(tol), _p(out))
    return out


def orders_from_pred(tree: Tree, pred, margin_q, margin_p, q_lo, q_hi, p_lo, p_hi, p_default, tgt_ctr=None):
    """Per-center QBX orders and per-box local-expansion orders from predictions (n_ctr, 2)."""
    pr = np.ascontiguousarray(pred, np.float32)
    tc = None if tgt_ctr is None else np.ascontiguousarray(tgt_ctr, np.int32)
    q = np.zeros(pr.shape[0], np.int32)
    pb = np.zeros(tree.n_boxes, np.int32)
    lib().orc_orders_from_pred(tree.handle, _p(pr), _p(tc), float(margin_q), float(margin_p), q_lo, q_hi, p_lo, p_hi,
                               p_default, _p(q), _p(pb))
    return q, pb


def refine_marks(which, src_xyz, ctr_xyz, ctr_r, elem, n_elem, elem_eta=None, eps=0.025):
    """Bisection marks per element (bool[n_elem]): which = 0, Algorithm 1 (a source strictly inside
    (1 - eps) r of a center; elem per center), which = 1, Algorithm 2 (a center within 0.375 eta_k of a
    source of element k; elem per source, elem_eta per element)."""
    s, c, r = _f64(src_xyz), _f64(ctr_xyz), _f64(ctr_r)
    e = np.ascontiguousarray(elem, np.int32)
    eta = _f64(np.zeros(n_elem) if elem_eta is None else elem_eta)
    out = np.zeros(max(n_elem, 1), np.uint8)
    lib().orc_refine_marks(int(which), _p(s), s.shape[1], _p(c), _p(r), c.shape[1], _p(e), _p(eta), int(n_elem),
                           float(eps), _p(out))
    return out[:n_elem].astype(bool)
