"""Autotuner for the evaluation's launch shape: the leaf size n_max of the octree (which trades
direct P2QBXL work against translation work) and the tile parameters of the tensor-core
translation kernels (qbx_lists_set_tiles).

Candidates are timed on the problem itself (or a representative subset of a batch) with CUDA
events on the current stream; the winner is cached in a JSON file keyed by the device, the
precision mode, the orders and the problem size class, so later runs reuse it.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import torch

from . import binding as B

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _key(kind, precision, q, p, n_src):
    dev = torch.cuda.get_device_name()
    return f"{kind}|{dev}|prec{precision}|q{q}|p{p}|src2^{int(round(math.log2(max(n_src, 1))))}"


def _time_forest(G, surfs, dens, q, p, precision, n_max, tiles, reps=2):
    cu = lambda a, dt=torch.float64: torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()  # noqa: E731
    trees, lists = [], []
    for s in surfs:
        T = B.qbx_build_tree(cu(s.src_xyz), cu(s.ctr_xyz), cu(s.ctr_r), cu(s.tgt_xyz), n_max=n_max)
        trees.append(T)
        lists.append(B.qbx_build_lists(T))
    F, FL = B.qbx_build_forest(trees, lists) if len(trees) > 1 else (trees[0], lists[0])
    off = F.offsets if len(trees) > 1 else {"ctr": [0]}
    args = (cu(np.concatenate([s.src_w for s in surfs])), cu(np.concatenate(dens)), None,
            cu(np.concatenate([s.src_n for s in surfs], axis=1)),
            cu(np.concatenate([s.tgt_ctr + off["ctr"][i] for i, s in enumerate(surfs)]).astype(np.int32),
               torch.int32))
    if tiles is not None:
        B.qbx_lists_set_tiles(FL, *tiles)
    out = B.qbx_eval(F, FL, *args, q, p, precision=precision)
    st = torch.cuda.current_stream()
    best = math.inf
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        B.qbx_eval(F, FL, *args, q, p, precision=precision, out=out)
        e1.record(st)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def _subset(surfs, dens, max_sources):
    """Surfaces spread over the size range (every k-th by size) holding at most max_sources sources."""
    order = np.argsort([s.n_src for s in surfs])
    pick, total = [], 0
    step = max(1, len(order) // 8)
    for i in order[::step]:
        if total + surfs[i].n_src > max_sources and pick:
            break
        pick.append(i)
        total += surfs[i].n_src
    return [surfs[i] for i in pick], [dens[i] for i in pick]


def tuned_n_max(G, surfs, dens, q, p, precision, default=64, candidates=(32, 48, 64, 96, 128),
                tile_candidates=((0, 0), (16, 48), (32, 64)), enabled=True, max_sources=300_000):
    """Leaf size and tensor-core tiles for evaluating `surfs` (list of synth surfaces) with the given
    orders and precision.  Returns {"n_max", "tiles", "source": "cache" | "tuned" | "default", ...}."""
    n_src = int(sum(s.n_src for s in surfs))
    key = _key("forest" if len(surfs) > 1 else "single", precision, q, p, n_src)
    db = _load()
    if key in db:
        return {**db[key], "source": "cache", "key": key}
    if not enabled:
        return {"n_max": default, "tiles": [0, 0], "source": "default", "key": key}
    sub_s, sub_d = _subset(surfs, dens, max_sources)
    timings = {}
    for nm in candidates:
        timings[str(nm)] = _time_forest(G, sub_s, sub_d, q, p, precision, nm, None)
    best_nm = int(min(timings, key=timings.get))
    tile_t = {}
    if precision == B.QBX_M2L_3XTF32:
        for tl in tile_candidates:
            tile_t[f"{tl[0]},{tl[1]}"] = _time_forest(G, sub_s, sub_d, q, p, precision, best_nm, tl)
    best_tiles = [int(v) for v in min(tile_t, key=tile_t.get).split(",")] if tile_t else [0, 0]
    rec = {"n_max": best_nm, "tiles": best_tiles, "timings_ms": timings, "tile_timings_ms": tile_t,
           "subset_sources": int(sum(s.n_src for s in sub_s))}
    db[key] = rec
    _store(db)
    return {**rec, "source": "tuned", "key": key}
