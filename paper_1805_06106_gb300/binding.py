"""Thin ctypes binding of libqbx (include/qbx.h).

Argument marshalling only: PyTorch CUDA tensors provide device memory and the
current stream; every step of the evaluation runs in the library's kernels.
There is no CPU fallback: loading fails loudly if the library cannot be built or
loaded.  Functions keep the C names.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

QBX_FP64, QBX_M2L_FP32, QBX_M2L_3XTF32 = 0, 1, 2
QBX_MIXED_M2L_ONLY, QBX_MIXED_M2QBXL_ONLY = 0x10, 0x20
QBX_TREE_LINF_TCR, QBX_TREE_LEVEL_RESTRICT = 1, 2
QBX_REFINE_INTERFERING, QBX_REFINE_QUAD_RES = 0, 1
LIST_NAMES = ("U", "V", "Wclose", "Wfar", "Xclose", "Xfar")
STAGE_NAMES = ("prep", "p2m_m2m", "m2l", "p2l", "l2l", "m2qbxl_mixed", "centers", "m2qbxl_reduce", "qbx_targets",
               "point_targets")


class QbxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libqbx error {code}: {msg}")
        self.code = code


class _TreeOpts(C.Structure):
    _fields_ = [("n_max", C.c_int), ("t_f", C.c_double), ("max_depth", C.c_int), ("flags", C.c_uint)]


class _TreeInfo(C.Structure):
    _fields_ = [("n_boxes", C.c_int64), ("n_levels", C.c_int64), ("n_src", C.c_int64), ("n_ctr", C.c_int64),
                ("n_tgt", C.c_int64), ("n_overfull", C.c_int64), ("root_center", C.c_double * 3),
                ("root_radius", C.c_double)]


class _Cost(C.Structure):
    _fields_ = [("count", C.c_int64 * 6), ("ops", C.c_double * 6), ("ops_stages", C.c_double),
                ("ops_total", C.c_double)]


class _EvalOpts(C.Structure):
    _fields_ = [("p_qbx", C.c_int), ("p_fmm", C.c_int), ("p_qbx_per_ctr", C.c_void_p),
                ("p_fmm_per_box", C.c_void_p), ("precision", C.c_int)]


_lib = None


def lib():
    """Load (building first if needed) libqbx.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P, I64 = C.c_void_p, C.c_int64
        L.qbx_build_tree.argtypes = [P, I64, P, P, I64, P, I64, C.POINTER(_TreeOpts), C.POINTER(P), P]
        L.qbx_tree_query.argtypes = [P, C.POINTER(_TreeInfo)]
        L.qbx_tree_export.argtypes = [P] * 9
        L.qbx_tree_free.argtypes = [P]
        L.qbx_tree_free.restype = None
        L.qbx_build_lists.argtypes = [P, C.POINTER(P), P]
        L.qbx_lists_nnz.argtypes = [P, C.c_int, C.POINTER(I64)]
        L.qbx_lists_export.argtypes = [P, C.c_int, P, P, P]
        L.qbx_lists_free.argtypes = [P]
        L.qbx_lists_free.restype = None
        L.qbx_assoc_targets.argtypes = [P, P, P, P, C.c_double, P, P, P]
        L.qbx_refine_marks.argtypes = [P, C.c_int, P, P, I64, C.c_double, P, P]
        L.qbx_lists_cost.argtypes = [P, C.c_int, C.c_int, C.POINTER(_Cost), P]
        L.qbx_eval.argtypes = [P, P, P, P, P, P, P, C.POINTER(_EvalOpts), P, P]
        L.qbx_eval_noalloc.argtypes = [P, P, P, P, P, P, P, C.POINTER(_EvalOpts), P, P]
        L.qbx_eval_order_sweep.argtypes = [P, P, P, P, P, P, P, C.POINTER(_EvalOpts), P, P]
        L.qbx_center_features.argtypes = [P, P, P, P, P, P, P, P]
        L.qbx_order_labels.argtypes = [P, C.c_int, P, I64, C.c_double, P, P]
        L.qbx_mlp_init.argtypes = [P, C.c_uint64, P]
        L.qbx_mlp_forward.argtypes = [P, P, I64, P, P]
        L.qbx_mlp_loss_grad.argtypes = [P, P, P, I64, P, P]
        L.qbx_mlp_train.argtypes = [P, P, P, P, P, I64, C.c_int, C.c_int, C.c_float, P, P]
        L.qbx_orders_from_mlp.argtypes = [P, P, P, P, C.c_float, C.c_float, C.c_int, C.c_int, C.c_int, C.c_int,
                                          C.c_int, P, P, P]
        L.qbx_orders_fallback.argtypes = [P, P, P, P, C.c_double, C.c_int, C.c_int, P, P, C.POINTER(I64), P]
        L.qbx_build_forest.argtypes = [C.c_int, P, P, C.POINTER(P), C.POINTER(P), P]
        L.qbx_forest_problems.argtypes = [P, C.POINTER(C.c_int)]
        L.qbx_forest_offsets.argtypes = [P, P]
        L.qbx_graph_create.argtypes = [P, P, P, P, P, P, P, C.POINTER(_EvalOpts), P, C.POINTER(P), P]
        L.qbx_graph_launch.argtypes = [P, P]
        L.qbx_graph_free.argtypes = [P]
        L.qbx_graph_free.restype = None
        L.qbx_lists_set_tiles.argtypes = [P, C.c_int, C.c_int]
        L.qbx_lists_set_wait.argtypes = [P, C.c_longlong, C.c_int]
        L.qbx_profile.argtypes = [P, C.c_int]
        L.qbx_profile_read.argtypes = [P, P]
        L.qbx_peak_flops.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double), P]
        L.qbx_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise QbxError(rc, lib().qbx_last_error().decode())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(x, dtype):
    if x is None:
        return None
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if x.dtype != dtype or not x.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} tensor")
    return x


def _ptr(x):
    return None if x is None else C.c_void_p(x.data_ptr())


class Tree:
    def __init__(self, handle):
        self.handle = handle
        info = _TreeInfo()
        _check(lib().qbx_tree_query(handle, C.byref(info)))
        self.info = info
        self.n_boxes = info.n_boxes

    def export(self):
        """Tree arrays as CUDA tensors (level, coords, parent, child, src/ctr/tgt owner)."""
        i = self.info
        dev = torch.device("cuda")
        out = dict(level=torch.empty(i.n_boxes, dtype=torch.int32, device=dev),
                   coords=torch.empty((i.n_boxes, 3), dtype=torch.int64, device=dev),
                   parent=torch.empty(i.n_boxes, dtype=torch.int32, device=dev),
                   child=torch.empty((i.n_boxes, 8), dtype=torch.int32, device=dev),
                   src_owner=torch.empty(i.n_src, dtype=torch.int32, device=dev),
                   ctr_owner=torch.empty(i.n_ctr, dtype=torch.int32, device=dev),
                   tgt_owner=torch.empty(i.n_tgt, dtype=torch.int32, device=dev))
        _check(lib().qbx_tree_export(self.handle, *[_ptr(out[k]) for k in ("level", "coords", "parent", "child",
                                                                            "src_owner", "ctr_owner", "tgt_owner")],
                                     _stream()))
        return out

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qbx_tree_free(self.handle)
            self.handle = None


class Lists:
    def __init__(self, handle, tree):
        self.handle = handle
        self.tree = tree  # keeps the tree alive while the lists exist

    def nnz(self, which):
        v = C.c_int64()
        _check(lib().qbx_lists_nnz(self.handle, which, C.byref(v)))
        return v.value

    def export(self):
        out = {}
        nb = self.tree.n_boxes
        for k, name in enumerate(LIST_NAMES):
            st = torch.empty(nb + 1, dtype=torch.int32, device="cuda")
            ix = torch.empty(max(self.nnz(k), 1), dtype=torch.int32, device="cuda")
            _check(lib().qbx_lists_export(self.handle, k, _ptr(st), _ptr(ix), _stream()))
            out[name] = (st, ix[: self.nnz(k)])
        return out

    def profile(self, enable=True):
        """Turn per-stage CUDA-event timing of later qbx_eval calls on or off."""
        _check(lib().qbx_profile(self.handle, 1 if enable else 0))

    def stage_ms(self):
        """Stage durations (ms) of the last profiled qbx_eval, keyed by STAGE_NAMES."""
        import numpy as np

        out = np.zeros(len(STAGE_NAMES))
        _check(lib().qbx_profile_read(self.handle, C.c_void_p(out.ctypes.data)))
        return dict(zip(STAGE_NAMES, out.tolist()))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qbx_lists_free(self.handle)
            self.handle = None


def qbx_build_tree(src_xyz, ctr_xyz, ctr_r, tgt_xyz, n_max=32, t_f=0.9, max_depth=40, linf_tcr=False,
                   level_restrict=False) -> Tree:
    """Octree with target confinement (Algorithm 4 Stage 1). Inputs: CUDA float64 (3, N) / (N,).
    linf_tcr / level_restrict select QBX_TREE_LINF_TCR / QBX_TREE_LEVEL_RESTRICT."""
    s, c, r, t = (_dev(x, torch.float64) for x in (src_xyz, ctr_xyz, ctr_r, tgt_xyz))
    flags = (QBX_TREE_LINF_TCR if linf_tcr else 0) | (QBX_TREE_LEVEL_RESTRICT if level_restrict else 0)
    opts = _TreeOpts(n_max, t_f, max_depth, flags)
    h = C.c_void_p()
    _check(lib().qbx_build_tree(_ptr(s), s.shape[1], _ptr(c), _ptr(r), c.shape[1], _ptr(t), t.shape[1],
                                C.byref(opts), C.byref(h), _stream()))
    return Tree(h)


def qbx_build_lists(tree: Tree) -> Lists:
    h = C.c_void_p()
    _check(lib().qbx_build_lists(tree.handle, C.byref(h), _stream()))
    return Lists(h, tree)


def qbx_assoc_targets(tree: Tree, src_danger_r, src_n=None, ctr_side=None, eps=0.05):
    """Target association (Algorithm 3) for every target of the tree: (tgt_ctr int32, -1 = none;
    flagged int8) on the device, input order.  src_n / ctr_side None: no side preference."""
    rd = _dev(src_danger_r, torch.float64)
    n = _dev(src_n, torch.float64)
    cs = _dev(ctr_side, torch.int8)
    nt = tree.info.n_tgt
    tc = torch.empty(nt, dtype=torch.int32, device="cuda")
    fl = torch.empty(nt, dtype=torch.int8, device="cuda")
    _check(lib().qbx_assoc_targets(tree.handle, _ptr(rd), _ptr(n), _ptr(cs), float(eps), _ptr(tc), _ptr(fl),
                                   _stream()))
    return tc, fl


def qbx_refine_marks(tree: Tree, which, elem, n_elem, elem_eta=None, eps=0.025):
    """Element marks of Algorithm 1 (which = QBX_REFINE_INTERFERING, elem per center) or Algorithm 2
    (QBX_REFINE_QUAD_RES, elem per source, elem_eta per element): uint8[n_elem] on the device."""
    e = _dev(elem, torch.int32)
    eta = _dev(elem_eta, torch.float64)
    out = torch.empty(max(int(n_elem), 1), dtype=torch.uint8, device="cuda")
    _check(lib().qbx_refine_marks(tree.handle, int(which), _ptr(e), _ptr(eta), int(n_elem), float(eps), _ptr(out),
                                  _stream()))
    return out[:int(n_elem)]


def qbx_lists_cost(lists: Lists, p_qbx, p_fmm) -> dict:
    """Modeled operation counts (Section 6.3) of an evaluation on these lists: per-list integer
    counts ("count"), per-list modeled operations ("ops"), the remaining stage terms and the total."""
    c = _Cost()
    _check(lib().qbx_lists_cost(lists.handle, int(p_qbx), int(p_fmm), C.byref(c), _stream()))
    return {"count": dict(zip(LIST_NAMES, list(c.count))), "ops": dict(zip(LIST_NAMES, list(c.ops))),
            "stages": c.ops_stages, "total": c.ops_total}


def qbx_eval(tree: Tree, lists: Lists, src_w, sigma, mu, src_n, tgt_ctr, p_qbx, p_fmm, p_qbx_per_ctr=None,
             p_fmm_per_box=None, precision=QBX_FP64, out=None):
    """pot = S[sigma] + D[mu] at every target (Algorithm 4 Stages 2-9)."""
    w = _dev(src_w, torch.float64)
    sg, m, n = _dev(sigma, torch.float64), _dev(mu, torch.float64), _dev(src_n, torch.float64)
    tc = _dev(tgt_ctr, torch.int32)
    qc, pb = _dev(p_qbx_per_ctr, torch.int8), _dev(p_fmm_per_box, torch.int8)
    if out is None:
        out = torch.empty(tc.shape[0], dtype=torch.float64, device=tc.device)
    opts = _EvalOpts(p_qbx, p_fmm, None if qc is None else qc.data_ptr(), None if pb is None else pb.data_ptr(),
                     precision)
    _check(lib().qbx_eval(tree.handle, lists.handle, _ptr(w), _ptr(sg), _ptr(m), _ptr(n), _ptr(tc), C.byref(opts),
                          _ptr(out), _stream()))
    return out


def qbx_eval_noalloc(tree: Tree, lists: Lists, src_w, sigma, mu, src_n, tgt_ctr, p_qbx, p_fmm, out,
                     p_qbx_per_ctr=None, p_fmm_per_box=None, precision=QBX_FP64):
    """qbx_eval for callers that cannot allocate device memory: the library takes its scratch
    from a fixed 48 MiB array, and `out` must be given."""
    w = _dev(src_w, torch.float64)
    sg, m, n = _dev(sigma, torch.float64), _dev(mu, torch.float64), _dev(src_n, torch.float64)
    tc = _dev(tgt_ctr, torch.int32)
    qc, pb = _dev(p_qbx_per_ctr, torch.int8), _dev(p_fmm_per_box, torch.int8)
    out = _dev(out, torch.float64)
    opts = _EvalOpts(p_qbx, p_fmm, None if qc is None else qc.data_ptr(), None if pb is None else pb.data_ptr(),
                     precision)
    _check(lib().qbx_eval_noalloc(tree.handle, lists.handle, _ptr(w), _ptr(sg), _ptr(m), _ptr(n), _ptr(tc),
                                  C.byref(opts), _ptr(out), _stream()))
    return out


def qbx_eval_order_sweep(tree: Tree, lists: Lists, src_w, sigma, mu, src_n, tgt_ctr, p_qbx, p_fmm,
                         precision=QBX_FP64):
    """Potentials with every QBX local truncated at each order 0..p_qbx: tensor (p_qbx+1, n_tgt)."""
    w = _dev(src_w, torch.float64)
    sg, m, n = _dev(sigma, torch.float64), _dev(mu, torch.float64), _dev(src_n, torch.float64)
    tc = _dev(tgt_ctr, torch.int32)
    out = torch.empty((p_qbx + 1, tc.shape[0]), dtype=torch.float64, device=tc.device)
    opts = _EvalOpts(p_qbx, p_fmm, None, None, precision)
    _check(lib().qbx_eval_order_sweep(tree.handle, lists.handle, _ptr(w), _ptr(sg), _ptr(m), _ptr(n), _ptr(tc),
                                      C.byref(opts), _ptr(out), _stream()))
    return out


# ---------------------------------------------------------------- learned orders

MLP_NPARAMS = 4610


def qbx_center_features(tree: Tree, lists: Lists, src_w, sigma, mu, src_n):
    """(n_ctr, 4) float32 features per center (input order)."""
    w = _dev(src_w, torch.float64)
    sg, m, n = _dev(sigma, torch.float64), _dev(mu, torch.float64), _dev(src_n, torch.float64)
    out = torch.empty((tree.info.n_ctr, 4), dtype=torch.float32, device="cuda")
    _check(lib().qbx_center_features(tree.handle, lists.handle, _ptr(w), _ptr(sg), _ptr(m), _ptr(n), _ptr(out),
                                     _stream()))
    return out


def qbx_order_labels(values, orders, tol):
    """values (K, n) float64 results at increasing orders (last = reference) -> (n,) int8 labels."""
    v = _dev(values.contiguous(), torch.float64)
    arr = (C.c_int * len(orders))(*orders)
    out = torch.empty(v.shape[1], dtype=torch.int8, device=v.device)
    _check(lib().qbx_order_labels(_ptr(v), len(orders), arr, v.shape[1], float(tol), _ptr(out), _stream()))
    return out


def qbx_mlp_init(seed=0):
    p = torch.empty(MLP_NPARAMS, dtype=torch.float32, device="cuda")
    _check(lib().qbx_mlp_init(_ptr(p), int(seed), _stream()))
    return p


def qbx_mlp_forward(params, x):
    x = _dev(x.contiguous(), torch.float32)
    y = torch.empty((x.shape[0], 2), dtype=torch.float32, device=x.device)
    _check(lib().qbx_mlp_forward(_ptr(_dev(params, torch.float32)), _ptr(x), x.shape[0], _ptr(y), _stream()))
    return y


def qbx_mlp_loss_grad(params, x, target):
    g = torch.empty(MLP_NPARAMS + 1, dtype=torch.float32, device="cuda")
    _check(lib().qbx_mlp_loss_grad(_ptr(_dev(params, torch.float32)), _ptr(_dev(x.contiguous(), torch.float32)),
                                   _ptr(_dev(target.contiguous(), torch.float32)), x.shape[0], _ptr(g), _stream()))
    return g[:-1], float(g[-1])


def qbx_mlp_train(params, adam_m, adam_v, x, target, steps, first_step, lr):
    loss = C.c_float()
    _check(lib().qbx_mlp_train(_ptr(_dev(params, torch.float32)), _ptr(_dev(adam_m, torch.float32)),
                               _ptr(_dev(adam_v, torch.float32)), _ptr(_dev(x.contiguous(), torch.float32)),
                               _ptr(_dev(target.contiguous(), torch.float32)), x.shape[0], steps, first_step,
                               float(lr), C.byref(loss), _stream()))
    return loss.value


def qbx_orders_from_mlp(tree: Tree, lists: Lists, pred, margin_q, margin_p, q_lo, q_hi, p_lo, p_hi, p_default,
                        tgt_ctr=None):
    """Per-center QBX orders and per-box local-expansion orders from network predictions; tgt_ctr
    (optional) marks point targets, whose boxes keep p_hi."""
    qc = torch.empty(tree.info.n_ctr, dtype=torch.int8, device="cuda")
    pb = torch.empty(tree.n_boxes, dtype=torch.int8, device="cuda")
    tc = _dev(tgt_ctr, torch.int32)
    _check(lib().qbx_orders_from_mlp(tree.handle, lists.handle, _ptr(_dev(pred.contiguous(), torch.float32)),
                                     _ptr(tc), float(margin_q), float(margin_p), q_lo, q_hi, p_lo, p_hi, p_default,
                                     _ptr(qc), _ptr(pb), _stream()))
    return qc, pb


def qbx_orders_fallback(tree: Tree, result, judge, tgt_ctr, tol, q_fix, p_fix, p_qbx_per_ctr, p_fmm_per_box):
    """Raise, in place, the orders of every center / box chain whose target misses the fixed-order
    judge by more than tol (absolute); returns the number of such targets."""
    n = C.c_int64()
    _check(lib().qbx_orders_fallback(tree.handle, _ptr(_dev(result, torch.float64)), _ptr(_dev(judge, torch.float64)),
                                     _ptr(_dev(tgt_ctr, torch.int32)), float(tol), int(q_fix), int(p_fix),
                                     _ptr(_dev(p_qbx_per_ctr, torch.int8)), _ptr(_dev(p_fmm_per_box, torch.int8)),
                                     C.byref(n), _stream()))
    return n.value


def qbx_lists_set_tiles(lists: Lists, m2l_kchunk=0, m2qbxl_kchunk=0):
    """Launch-shape hints of the tensor-core translation kernels (0 = library default)."""
    _check(lib().qbx_lists_set_tiles(lists.handle, int(m2l_kchunk), int(m2qbxl_kchunk)))


def qbx_lists_set_wait(lists: Lists, limit_cycles=0, probe_step=-1):
    """Tensor-core pipeline wait limit (cycles; 0 = default) and failure-path probe step (-1 = off)."""
    _check(lib().qbx_lists_set_wait(lists.handle, int(limit_cycles), int(probe_step)))


# ---------------------------------------------------------------- batched problems and graphs


def qbx_build_forest(trees, lists):
    """Concatenate built trees and their lists into one forest: returns (Tree, Lists).

    The returned Tree has `offsets` (dict of int64 prefix sums per problem: boxes, src, ctr, tgt)."""
    n = len(trees)
    if n != len(lists) or n == 0:
        raise ValueError("need matching, non-empty lists of trees and lists")
    th = (C.c_void_p * n)(*[t.handle for t in trees])
    lh = (C.c_void_p * n)(*[x.handle for x in lists])
    fh, flh = C.c_void_p(), C.c_void_p()
    _check(lib().qbx_build_forest(n, th, lh, C.byref(fh), C.byref(flh), _stream()))
    F = Tree(fh)
    FL = Lists(flh, F)
    off = (C.c_int64 * (4 * (n + 1)))()
    _check(lib().qbx_forest_offsets(fh, off))
    vals = list(off)
    F.offsets = {k: vals[i * (n + 1):(i + 1) * (n + 1)] for i, k in enumerate(("boxes", "src", "ctr", "tgt"))}
    F.n_problems = n
    return F, FL


class Graph:
    """A captured qbx_eval (qbx_graph_create); launch() replays it on the current stream."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep  # tensors whose pointers are baked into the graph

    def launch(self):
        _check(lib().qbx_graph_launch(self.handle, _stream()))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qbx_graph_free(self.handle)
            self.handle = None


def qbx_graph_create(tree: Tree, lists: Lists, src_w, sigma, mu, src_n, tgt_ctr, p_qbx, p_fmm, out,
                     p_qbx_per_ctr=None, p_fmm_per_box=None, precision=QBX_FP64) -> Graph:
    """Capture one evaluation into a CUDA graph (needs a non-default current stream); `out` receives
    the potentials of every replay.  The graph keeps references to every tensor it reads."""
    w = _dev(src_w, torch.float64)
    sg, m, n = _dev(sigma, torch.float64), _dev(mu, torch.float64), _dev(src_n, torch.float64)
    tc = _dev(tgt_ctr, torch.int32)
    qc, pb = _dev(p_qbx_per_ctr, torch.int8), _dev(p_fmm_per_box, torch.int8)
    out = _dev(out, torch.float64)
    opts = _EvalOpts(p_qbx, p_fmm, None if qc is None else qc.data_ptr(), None if pb is None else pb.data_ptr(),
                     precision)
    h = C.c_void_p()
    _check(lib().qbx_graph_create(tree.handle, lists.handle, _ptr(w), _ptr(sg), _ptr(m), _ptr(n), _ptr(tc),
                                  C.byref(opts), _ptr(out), C.byref(h), _stream()))
    return Graph(h, (tree, lists, w, sg, m, n, tc, qc, pb, out))


QBX_PEAK_FP64, QBX_PEAK_FP32 = 0, 1


def qbx_peak_flops(kind, reps=5):
    """Measured FMA throughput of the device in flop/s (kind QBX_PEAK_FP64 or QBX_PEAK_FP32)."""
    v = C.c_double()
    _check(lib().qbx_peak_flops(int(kind), int(reps), C.byref(v), _stream()))
    return v.value


def library_path() -> str:
    return os.path.abspath(_build.LIB)
