"""Benchmark of the GB300 GIGAQBX evaluation (Algorithm 4, Stages 2-9).

Workload (default): the star surface r = 1 + 0.3 Re Y_6^3 with 8,000 curved
triangles x 15 nodes (120,000 sources), two QBX centers per node at radius
eta_k/2 (240,000 centers, one on-surface target each) plus 10,000 volume points
in [-2,2]^3 associated by Algorithm 3; densities sigma = d_n u and mu = -u for
u = 1/|x - (3,1,2)| (Green's formula S(d_n u) - D(u)); p_qbx = 7, p_fmm = 15,
t_f = 0.9.  A step is one qbx_eval (every stage of the evaluation) with the tree
and lists built beforehand, as in repeated evaluation inside an iterative solver.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gpu,reference}]

--impl reference times the FP64 CPU oracle (the reference arm) on a bounded
sample of the same workload.  Under torchrun each rank evaluates its own replica
(the path needs no exchange between GPUs).  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QBX target evals/s at 1e-6 rel err: learned+mixed vs plain FP64 GIGAQBX"
P_QBX, P_FMM, T_F = 7, 15, 0.9
TOL = 1e-6            # acceptance: normwise relative l-infinity distance to the fixed-order FP64 result
N_MAX = 256           # leaf size of plain FP64 (best of its n_max sweep)
N_MAX_MIXED = 48      # leaf size of the mixed-precision mode (profiles/nmax_sweep_star8k.md)
N_VOLUME = 10000
FP64_PEAK_TFLOPS = 1.258  # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (1.25 TFLOP/s nominal)
L2_FLUSH_BYTES = 512 << 20


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# Named single-surface workloads: (faces subdivided n x n, shape, density, (p_qbx, p_fmm), volume points)
WORKLOADS = {
    # 8,000 curved triangles (120,000 sources): S[d_n u] - D[u], Green's formula
    "star8k": (20, "Y63", "greens", (7, 15), 10000),
    # 40,500 curved triangles (607,500 sources): the precision variant of the same star
    "star40k": (45, "Y63", "greens", (7, 15), 10000),
    # 79,380 curved triangles (1,190,700 sources): the learned-order surface, random Y_n^m density
    "star79k": (63, "Y84Y52", "random", (8, 16), 0),
}


def make_workload(n_sub=20, name="star8k"):
    from synth import greens_density, make_surface, random_harmonic_density, star_radius, volume_targets
    from synth.surfaces import STAR_Y63, STAR_Y84_Y52

    _, shape, dens, _, nvol = WORKLOADS[name]
    s = make_surface(n_sub, star_radius(STAR_Y63 if shape == "Y63" else STAR_Y84_Y52))
    if dens == "greens":
        u, dudn = greens_density(s)
        sigma, mu = dudn, -u
    else:
        sigma, mu = random_harmonic_density(s, 10, 4), None
    if nvol:
        vt, vc, vflag = volume_targets(s, nvol, seed=2)
        t = np.concatenate([s.tgt_xyz, vt], axis=1)
        tc = np.concatenate([s.tgt_ctr, vc]).astype(np.int32)
    else:
        t, tc, vflag = s.tgt_xyz, s.tgt_ctr.astype(np.int32), np.zeros(0, bool)
    return s, sigma, mu, t, tc, vflag


# ------------------------------------------------------------------ algorithmic work model


def _tri(p):
    return (p + 1) * (p + 2) // 2


def _l2qbxl_macs(P, Q):
    n_mac = 0
    for n in range(P + 1):
        for m in range(-n, n + 1):
            for k in range(min(n, Q) + 1):
                j = n - k
                n_mac += sum(1 for l in range(k + 1) if abs(m - l) <= j)
    return n_mac


def center_kernel_flops(P, Q, n_direct_pairs, n_wfar_pairs, n_centers, dipole=True):
    """FP64 flops of the formulas the fused center kernel evaluates (mul, add = 1; fused mul-add = 2).

    direct pair: 16 (geometry, 1/r^2, 1/r) + 8 per irregular harmonic entry up to order
    K = Q + dipole + per output coefficient 4 (charge) or 22 (charge + dipole);
    List 3 far pair: 8 per harmonic up to P+Q + 8 per complex MAC over (P+1)^2 x ntri(Q);
    L2QBXL per center: 8 per harmonic up to P + 8 per complex MAC of the shift.
    """
    K = Q + (1 if dipole else 0)
    f_pair = 16 + 8 * (_tri(K) - 1) + (22 if dipole else 4) * _tri(Q)
    f_wfar = 8 * _tri(P + Q) + 8 * (P + 1) ** 2 * _tri(Q) + 2 * (P + 1) ** 2
    f_l2q = 8 * _tri(P) + 8 * _l2qbxl_macs(P, Q)
    return f_pair * n_direct_pairs + f_wfar * n_wfar_pairs + f_l2q * n_centers, f_pair


def list_work(G, T, L):
    """Per-launch work units of the center kernel and the paper's modeled operation counts."""
    tr = {k: v.cpu().numpy() for k, v in T.export().items()}
    ls = {k: (a.cpu().numpy(), b.cpu().numpy()) for k, (a, b) in L.export().items()}
    nb = T.n_boxes
    nsrc = np.bincount(tr["src_owner"], minlength=nb).astype(np.int64)
    nctr = np.bincount(tr["ctr_owner"], minlength=nb).astype(np.int64)

    def per_box_sum(name, weight):
        st, ix = ls[name]
        cs = np.concatenate([[0], np.cumsum(weight[ix])])
        return cs[st[1:]] - cs[st[:-1]]

    direct_src = per_box_sum("U", nsrc) + per_box_sum("Wclose", nsrc) + per_box_sum("Xclose", nsrc)
    wfar = np.diff(ls["Wfar"][0]).astype(np.int64)
    n_direct = int(np.sum(direct_src * nctr))
    n_wfar = int(np.sum(wfar * nctr))
    # modeled operation counts (Table ilist-operation-counts), n_t = centers of the target box
    q2, p3, p2 = P_QBX ** 2, P_FMM ** 3, P_FMM ** 2
    sub_src = np.zeros(nb, np.int64)
    par = tr["parent"]
    for b in range(nb - 1, -1, -1):
        sub_src[b] += nsrc[b]
        if par[b] >= 0:
            sub_src[par[b]] += sub_src[b]
    modeled = {
        "U": q2 * float(np.sum(per_box_sum("U", nsrc) * nctr)),
        "V": p3 * float(len(ls["V"][1])),
        "Wclose": q2 * float(np.sum(per_box_sum("Wclose", nsrc) * nctr)),
        "Wfar": p3 * float(n_wfar),
        "Xclose": q2 * float(np.sum(per_box_sum("Xclose", nsrc) * nctr)),
        "Xfar": p2 * float(np.sum(per_box_sum("Xfar", sub_src))),
    }
    return n_direct, n_wfar, modeled


def kernel_traffic():
    """DRAM bytes per launch of the center kernel from the committed ncu summary, or None when the
    kernel source changed since those counters were taken."""
    import hashlib

    prof_path = os.path.join(ROOT, "profiles", "traffic_centers_star8k.json")
    try:
        rec = json.load(open(prof_path))
        src = b"".join(open(os.path.join(ROOT, "paper_1805_06106_gb300", "csrc", f), "rb").read()
                       for f in ("eval.cu", "harmonics.cuh"))
        if hashlib.sha256(src).hexdigest()[:16] != rec.get("source_sha256_16"):
            return None
        return rec.get("bytes_per_launch")
    except (OSError, ValueError):
        return None


def library_launches(nlev, mixed):
    """Kernels of libqbx per evaluation: prep (3), P2M, M2M per level, M2L (1, or convert + GEMM +
    reduce), P2L, L2L per level, M2QBXL (0, or operator + GEMM), centers (+ List 3 far reduce),
    QBX targets, point targets (count, scan, fill, M2P pairs, P2P/L2P)."""
    return 3 + 1 + (nlev - 1) + (3 if mixed else 1) + 1 + (nlev - 1) + (2 if mixed else 0) + (3 if mixed else 2) + 5


# ------------------------------------------------------------------ clocks


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle baseline


def cpu_oracle_sample(n_sub=3):
    """Oracle FMM (Algorithm 4, serial FP64) on a bounded sample: the same surface family,
    densities and orders at 20 n_sub^2 elements (180 elements for the default n_sub = 3)."""
    import oracle as O
    from synth import greens_density, make_surface, star_radius
    from synth.surfaces import STAR_Y63

    s = make_surface(n_sub, star_radius(STAR_Y63))
    u, dudn = greens_density(s)
    t0 = time.perf_counter()
    T = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, s.tgt_xyz, n_max=N_MAX_MIXED, t_f=T_F)
    L = O.build_lists(T)
    t1 = time.perf_counter()
    O.fmm_eval(T, L, s.src_xyz, s.src_w, dudn, -u, s.src_n, s.ctr_xyz, s.tgt_xyz, s.tgt_ctr, P_QBX, P_FMM)
    t2 = time.perf_counter()
    n = s.n_ctr
    return {"value": n / (t2 - t1), "unit": "QBX target evals/s", "cores": 1, "kind": "oracle",
            "sample": f"serial FP64 oracle Algorithm 4 (Stages 2-9) on the same star family at {s.n_elem} elements "
                      f"({s.n_src} sources, {n} QBX targets), p_qbx={P_QBX}, p_fmm={P_FMM}, n_max={N_MAX_MIXED}; "
                      f"{t2 - t1:.1f} s eval + {t1 - t0:.2f} s tree/lists"}


def run_reference(args):
    ws, rank, _ = _dist_env()
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        cpu_oracle_sample(1)  # untimed warm-up on the smallest member of the family
    for _ in range(args.steps):
        vals.append(cpu_oracle_sample(2))
    v = statistics.median([x["value"] for x in vals])
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "QBX target evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "star r=1+0.3ReY63, 80 curved triangles x 15 nodes (oracle sample of the 120k-source star family)",
                       "p_qbx": P_QBX, "p_fmm": P_FMM, "n_max": N_MAX_MIXED, "t_f": T_F},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "QBX target evals/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm


def _measure(G, torch, dev, stream, geo, ev_in, n_out, n_max, prec, steps, warmup, want_clock, local,
             orders=None, rank_sync=None):
    """Build tree and lists for n_max, warm up, then time `steps` evaluations (CUDA events on the
    launching stream, L2 flushed between steps).  Returns timings, stage times and the result."""
    torch.cuda.synchronize()
    tb0 = time.perf_counter()
    T = G.qbx_build_tree(*geo, n_max=n_max, t_f=T_F)
    torch.cuda.synchronize()
    tb1 = time.perf_counter()
    L = G.qbx_build_lists(T)
    torch.cuda.synchronize()
    tb2 = time.perf_counter()
    pot = torch.empty(n_out, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    kw = dict(out=pot, precision=prec)
    if orders is not None:
        kw.update(orders(T, L))

    def step(inputs):
        G.qbx_eval(T, L, *inputs, P_QBX, P_FMM, **kw)

    L.profile(True)
    for _ in range(max(warmup, 3)):
        step(ev_in)
    torch.cuda.synchronize()
    ref = pot.clone()
    stage_tot = {k: 0.0 for k in G.STAGE_NAMES}
    step_ms = []
    if rank_sync:
        rank_sync()
    torch.cuda.synchronize()
    clk = ClockSampler(local) if want_clock else None
    if clk:
        clk.__enter__()
    try:
        for _ in range(steps):
            flush.fill_(1)  # L2 flush between timed iterations (outside the timed events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(ev_in)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            for k, v in L.stage_ms().items():
                stage_tot[k] += v
    finally:
        if clk:
            clk.__exit__(None, None, None)
    torch.cuda.synchronize()
    det = bool(torch.equal(pot, ref))
    L.profile(False)
    return dict(T=T, L=L, pot=ref, step_ms=step_ms, stage_ms={k: v / steps for k, v in stage_tot.items()},
                det=det, clk=clk, step=step, flush=flush, pot_buf=pot, tree_ms=1e3 * (tb1 - tb0),
                lists_ms=1e3 * (tb2 - tb1))


def learned_setup(G, n_max):
    """Train the order network on sweeps of configs 1-2 geometries (sphere and the Y_6^3 star at
    small sizes; Re Y_2^1, Green's-formula and random-harmonic densities), calibrate its margins."""
    from paper_1805_06106_gb300 import learned
    from synth import greens_density, make_surface, random_harmonic_density, real_ylm, star_radius
    from synth.surfaces import STAR_Y63

    t0 = time.perf_counter()
    samples = []
    for n, shape, seed in ((3, None, 11), (3, STAR_Y63, 12), (4, None, 13), (4, STAR_Y63, 14)):
        srf = make_surface(n) if shape is None else make_surface(n, star_radius(shape))
        if shape is None:
            samples.append(learned.sweep_samples(srf, real_ylm(2, 1, srf.src_xyz), None, P_QBX, P_FMM, n_max, TOL))
        else:
            uu, du = greens_density(srf)
            samples.append(learned.sweep_samples(srf, du, -uu, P_QBX, P_FMM, n_max, TOL))
        samples.append(learned.sweep_samples(srf, random_harmonic_density(srf, 10, seed), None, P_QBX, P_FMM, n_max,
                                             TOL))
    params, losses = learned.train(samples, steps=1000)
    mq, mp = learned.calibrate(params, samples)
    return params, (mq, mp), {"train_samples": int(sum(x.x.shape[0] for x in samples)), "final_loss": losses[-1],
                              "margins": [mq, mp], "setup_s": time.perf_counter() - t0}


def run_gpu(args):
    import torch

    ws, rank, local = _dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1805_06106_gb300 as G

    s, sigma, mu, t, tc, vflag = make_workload(args.n_sub, args.workload)
    n_qbx_tgt = int(np.sum(tc >= 0))
    n_pt_tgt = int(np.sum(tc < 0))

    def cu(a, dt=torch.float64):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dt).to(dev)

    precs = {"fp64": G.QBX_FP64, "fp32": G.QBX_M2L_FP32, "3xtf32": G.QBX_M2L_3XTF32,
             "learned": G.QBX_M2L_3XTF32 if args.mixed_form == "3xtf32" else G.QBX_M2L_FP32}
    mode = args.precision
    n_max = args.n_max if args.n_max else (N_MAX_MIXED if mode != "fp64" else N_MAX)
    orders_fn, learned_info = None, None
    if mode == "learned":
        from paper_1805_06106_gb300 import learned

        params, (mq, mp), learned_info = learned_setup(G, n_max)

        def orders_fn(T, L):
            w_, sg_, mu_, n_ = (cu(s.src_w), cu(sigma), None if mu is None else cu(mu), cu(s.src_n))
            qc, pb = learned.predict_orders(T, L, params, w_, sg_, mu_, n_, q_range=(2, P_QBX), p_range=(4, P_FMM),
                                            margin_q=mq, margin_p=mp, p_default=P_FMM,
                                            tgt_ctr=cu(tc, torch.int32))
            qn, pn = qc.cpu().numpy().astype(int), pb.cpu().numpy().astype(int)
            learned_info["mean_p_qbx"] = float(qn.mean())
            learned_info["mean_p_fmm_box"] = float(pn.mean())
            learned_info["qbx_order_work_vs_fixed"] = float(np.sum((qn + 1) * (qn + 2)) /
                                                            (qn.size * (P_QBX + 1) * (P_QBX + 2)))
            learned_info["fmm_order_work_vs_fixed"] = float(np.sum((pn + 1) ** 3) / (pn.size * (P_FMM + 1) ** 3))
            return dict(p_qbx_per_ctr=qc, p_fmm_per_box=pb)
    sync = (lambda: torch.distributed.barrier()) if ws > 1 else None

    def max_over_ranks(x):
        if ws == 1:
            return x
        tt = torch.tensor([x], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        return float(tt.item())

    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        geo = [cu(s.src_xyz), cu(s.ctr_xyz), cu(s.ctr_r), cu(t)]
        ev_in = (cu(s.src_w), cu(sigma), None if mu is None else cu(mu), cu(s.src_n), cu(tc, torch.int32))
        main = _measure(G, torch, dev, stream, geo, ev_in, t.shape[1], n_max, precs[mode], args.steps, args.warmup,
                        True, local, orders=orders_fn, rank_sync=sync)
        total_ms = max_over_ranks(float(sum(main["step_ms"])))
        ms_per_step = total_ms / args.steps
        value = ws * n_qbx_tgt * args.steps / (total_ms * 1e-3)

        # end to end through the public API: pinned host inputs in, potentials out
        host_in = [None if x is None else x.cpu().pin_memory() for x in ev_in]
        host_out = torch.empty(t.shape[1], dtype=torch.float64).pin_memory()
        dev_in = [None if x is None else torch.empty_like(x) for x in ev_in]
        h2d = sum(x.numel() * x.element_size() for x in host_in if x is not None)
        d2h = host_out.numel() * host_out.element_size()
        n_e2e = max(1, min(args.steps, 5))
        torch.cuda.synchronize()
        e2e_ms = []
        for _ in range(n_e2e):
            main["flush"].fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for d, h in zip(dev_in, host_in):
                if d is not None:
                    d.copy_(h, non_blocking=True)
            main["step"](dev_in)
            host_out.copy_(main["pot_buf"], non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            e2e_ms.append(e0.elapsed_time(e1))
        e2e_value = ws * n_qbx_tgt * n_e2e / (max_over_ranks(float(sum(e2e_ms))) * 1e-3)
        e2e_ok = bool(torch.equal(host_out.to(dev), main["pot"]))

        plain = None
        err_vs_fp64 = None
        if mode != "fp64":
            # accuracy of the mixed result against FP64 on the same tree and lists (untimed)
            T, L = main["T"], main["L"]
            ref64 = G.qbx_eval(T, L, *ev_in, P_QBX, P_FMM)
            err_vs_fp64 = float((main["pot"] - ref64).abs().max() / ref64.abs().max())
            if learned_info is not None:
                learned_info["within_tol_of_fixed_fp64"] = err_vs_fp64 <= TOL
        if mode != "fp64" and not args.no_fp64_baseline:
            # plain FP64 GIGAQBX at its own tuned leaf size, timed the same way
            base = _measure(G, torch, dev, stream, geo, ev_in, t.shape[1], N_MAX, G.QBX_FP64, args.fp64_steps,
                            args.warmup, False, local, rank_sync=sync)
            b_total = max_over_ranks(float(sum(base["step_ms"])))
            plain = {"value": ws * n_qbx_tgt * args.fp64_steps / (b_total * 1e-3), "ms_per_step": b_total / args.fp64_steps,
                     "n_max": N_MAX, "steps": args.fp64_steps, "stage_ms": base["stage_ms"]}

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    T, L = main["T"], main["L"]
    n_direct, n_wfar, modeled = list_work(G, T, L)
    flops, f_pair = center_kernel_flops(P_FMM, P_QBX, n_direct, 0 if mode != "fp64" else n_wfar, T.info.n_ctr,
                                        dipole=mu is not None)
    centers_ms = main["stage_ms"]["centers"]
    achieved = flops / (centers_ms * 1e-3) / 1e12
    nlev = int(T.info.n_levels)
    launches = library_launches(nlev, mode != "fp64")
    line = {
        "metric": METRIC, "value": value, "unit": "QBX target evals/s", "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if mode == "fp64" else (
            "f64 (List 2 M2L and List 3 far M2QBXL products in f32)" if precs[mode] == G.QBX_M2L_FP32 else
            "f64 (List 2 M2L and List 3 far M2QBXL products as split-tf32 tensor-core MMAs, f32 accumulation)"),
        "data": "synthetic",
        "config": {"workload": (f"{args.workload}: star r=1+0.3ReY63, {s.n_elem} curved triangles x 15 nodes: "
                                f"S[d_n u] - D[u] at {s.n_ctr} on-surface QBX targets + {n_pt_tgt} volume points"
                                if WORKLOADS[args.workload][1] == "Y63" else
                                f"{args.workload}: star r=1+0.25ReY84+0.15ReY52, {s.n_elem} curved triangles x 15 "
                                f"nodes: S[sigma], sigma = sum of N(0,1) Y_n^m (n<=10), at {s.n_ctr} on-surface QBX "
                                f"targets"),
                   "mode": {"fp64": "plain FP64 GIGAQBX, fixed orders",
                            "fp32": "mixed precision (FP32 translation products), fixed orders",
                            "3xtf32": "mixed precision (split-TF32 tensor-core translation products), fixed orders",
                            "learned": "learned orders + mixed precision (" + (
                                "split-TF32 tensor-core" if args.mixed_form == "3xtf32" else "FP32")
                            + " translation products)"}[mode],
                   "p_qbx": P_QBX, "p_fmm": P_FMM, "n_max": n_max, "t_f": T_F, "n_src": int(s.n_src),
                   "n_ctr": int(s.n_ctr), "n_qbx_targets": n_qbx_tgt, "n_point_targets": n_pt_tgt,
                   "n_flagged": int(vflag.sum()), "n_boxes": int(T.n_boxes), "n_levels": nlev,
                   "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "tree_build_ms": main["tree_ms"], "lists_build_ms": main["lists_ms"]},
        "stage_ms": main["stage_ms"],
        "modeled_ops": modeled,
        "deterministic": main["det"],
        "e2e": {"value": e2e_value, "unit": "QBX target evals/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "matches_device_result": e2e_ok},
        "gpu_launches": launches * args.steps,
        "roofline": {"kernel": "k_centers (L2QBXL + direct P2QBXL" + (", List 3 far M2QBXL" if mode == "fp64" else "")
                               + ", FP64)", "bound": "alu",
                     "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": kernel_traffic(),
                     "flops_per_launch": flops, "flops_per_direct_pair": f_pair, "direct_pairs": n_direct,
                     "wfar_pairs": n_wfar, "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz "
                                                          "(nominal 1.25 TFLOP/s; 1.195 measured by an FMA-chain probe)"},
        "clocks": main["clk"].summary(),
    }
    if learned_info is not None:
        line["learned_orders"] = learned_info
    if err_vs_fp64 is not None:
        line["rel_err_vs_fp64_same_tree"] = err_vs_fp64
    if plain is not None:
        line["plain_fp64"] = plain
        line["speedup_vs_plain_fp64"] = value / plain["value"]
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample()
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def forest_inputs(G, torch, dev, surfs, dens, n_max, t_tgt=None):
    """Trees, lists and the forest of many surfaces; concatenated evaluation inputs (single layer)."""
    def cu(a, dt=torch.float64):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dt).to(dev)

    trees, lists = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in surfs:
        T = G.qbx_build_tree(cu(s.src_xyz), cu(s.ctr_xyz), cu(s.ctr_r), cu(s.tgt_xyz), n_max=n_max, t_f=T_F)
        trees.append(T)
        lists.append(G.qbx_build_lists(T))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    F, FL = G.qbx_build_forest(trees, lists)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    off = F.offsets
    w = cu(np.concatenate([s.src_w for s in surfs]))
    sg = cu(np.concatenate(dens))
    nrm = cu(np.concatenate([s.src_n for s in surfs], axis=1))
    tc = cu(np.concatenate([s.tgt_ctr + off["ctr"][i] for i, s in enumerate(surfs)]).astype(np.int32), torch.int32)
    return dict(trees=trees, lists=lists, F=F, FL=FL, ev=(w, sg, None, nrm, tc), build_ms=1e3 * (t1 - t0),
                forest_ms=1e3 * (t2 - t1))


def run_batched(args):
    """Many surfaces of uneven size in one forest: learned orders + split-TF32 tensor-core
    translations replayed as one CUDA graph, against plain FP64 on the same surfaces."""
    import torch

    import paper_1805_06106_gb300 as G
    from paper_1805_06106_gb300 import autotune, learned
    from synth import batched_specs, make_surface, random_harmonic_density, star_radius

    from paper_1805_06106_gb300 import dist as D

    ws, rank, local = D.env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    all_specs = batched_specs(args.batch, seed=5)
    # the surfaces are independent: split them over the ranks by cost (sources), no exchange
    shard = D.lpt_shards([300 * n * n for n, _, _ in all_specs], ws)[rank]
    specs = [all_specs[i] for i in shard]
    t0 = time.perf_counter()
    surfs = [make_surface(n, star_radius(terms)) for n, terms, _ in specs]
    dens = [random_harmonic_density(s, 10, seed) for s, (_, _, seed) in zip(surfs, specs)]
    synth_s = time.perf_counter() - t0
    n_qbx_rank = int(sum(s.n_ctr for s in surfs))
    n_qbx = int(D.sum_over_ranks(n_qbx_rank, device=dev))
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        tuned = autotune.tuned_n_max(G, surfs, dens, P_QBX, P_FMM, G.QBX_M2L_3XTF32, default=N_MAX_MIXED,
                                     candidates=(32, 48, 64, 96), enabled=not args.no_tune)
        n_max = args.n_max or tuned["n_max"]
        fi = forest_inputs(G, torch, dev, surfs, dens, n_max)
        F, FL, ev = fi["F"], fi["FL"], fi["ev"]
        params, (mq, mp), info = learned_setup(G, n_max)
        # features per surface (each normalised by its own densities), orders on the forest
        preds = []
        for i, (T, L) in enumerate(zip(fi["trees"], fi["lists"])):
            o = F.offsets["src"]
            sl = slice(o[i], o[i + 1])
            feats = G.qbx_center_features(T, L, ev[0][sl].contiguous(), ev[1][sl].contiguous(), None,
                                          ev[3][:, sl].contiguous())
            preds.append(G.qbx_mlp_forward(params, feats))
        qc, pb = G.qbx_orders_from_mlp(F, FL, torch.cat(preds), mq, mp, 2, P_QBX, 4, P_FMM, P_FMM, tgt_ctr=ev[4])
        pot = torch.empty(int(F.info.n_tgt), dtype=torch.float64, device=dev)
        graph = G.qbx_graph_create(F, FL, *ev, P_QBX, P_FMM, pot, p_qbx_per_ctr=qc, p_fmm_per_box=pb,
                                   precision=G.QBX_M2L_3XTF32)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
        for _ in range(max(args.warmup, 3)):
            graph.launch()
        torch.cuda.synchronize()
        res = pot.clone()
        times = []
        D.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.__enter__()
        try:
            for _ in range(args.steps):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                graph.launch()
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
        finally:
            clk.__exit__(None, None, None)
        det = bool(torch.equal(pot, res))
        # end to end: pinned host densities in, potentials out, around the graph replay
        h_sig = ev[1].cpu().pin_memory()
        h_out = torch.empty_like(pot, device="cpu").pin_memory()
        e2e = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ev[1].copy_(h_sig, non_blocking=True)
            graph.launch()
            h_out.copy_(pot, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            e2e.append(e0.elapsed_time(e1))
        # plain FP64 on the same surfaces at its own leaf size, and FP64 at the learned run's tree
        ref_same = G.qbx_eval(F, FL, *ev, P_QBX, P_FMM)
        torch.cuda.synchronize()
        errs = []
        for i in range(len(surfs)):
            o = F.offsets["tgt"]
            a, b = res[o[i]:o[i + 1]], ref_same[o[i]:o[i + 1]]
            errs.append(float((a - b).abs().max() / b.abs().max()))
        build_ms, forest_ms = fi["build_ms"], fi["forest_ms"]
        del fi
        fp = forest_inputs(G, torch, dev, surfs, dens, N_MAX)
        ptmp = torch.empty_like(pot)
        G.qbx_eval(fp["F"], fp["FL"], *fp["ev"], P_QBX, P_FMM, out=ptmp)
        torch.cuda.synchronize()
        pt = []
        for _ in range(args.fp64_steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G.qbx_eval(fp["F"], fp["FL"], *fp["ev"], P_QBX, P_FMM, out=ptmp)
            e1.record(stream)
            e1.synchronize()
            pt.append(e0.elapsed_time(e1))
    ms = D.max_over_ranks(statistics.mean(times), device=dev)
    value = n_qbx / (ms * 1e-3)
    plain = n_qbx / (D.max_over_ranks(statistics.mean(pt), device=dev) * 1e-3)
    e2e_ms = D.max_over_ranks(statistics.mean(e2e), device=dev)
    errs_max = D.max_over_ranks(max(errs), device=dev)
    qn, pn = qc.cpu().numpy().astype(int), pb.cpu().numpy().astype(int)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": "QBX target evals/s", "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if ws > 1 else "weak",
        "vs_baseline": None,
        "dtype": "f64 (List 2 M2L and List 3 far M2QBXL products as split-tf32 tensor-core MMAs, f32 accumulation)",
        "data": "synthetic",
        "config": {"workload": f"{len(surfs)} star surfaces r=1+a ReY_k^(k/2), k in 2..10, a in [0.1,0.4], "
                               f"lognormal sizes ({int(sum(s.n_src for s in surfs))} sources, {n_qbx} QBX targets), "
                               "random Y_n^m (n<=10) single-layer densities; one forest, one CUDA graph",
                   "p_qbx": P_QBX, "p_fmm": P_FMM, "n_max": n_max, "n_max_source": tuned["source"], "t_f": T_F,
                   "sizes_src": [300 * n * n for n, _, _ in all_specs], "n_boxes_rank0": int(F.n_boxes),
                   "parallelism": f"surfaces split over {ws} GPUs by cost (LPT), no exchange" if ws > 1
                   else "single GPU",
                   "l2": "flushed between timed steps (512 MiB write)", "synth_s": synth_s,
                   "tree_lists_build_ms": build_ms, "forest_build_ms": forest_ms},
        "e2e": {"value": n_qbx / (e2e_ms * 1e-3), "unit": "QBX target evals/s",
                "h2d_bytes_per_step": int(h_sig.numel() * 8), "d2h_bytes_per_step": int(h_out.numel() * 8)},
        "gpu_launches": library_launches(int(F.info.n_levels), True) * args.steps, "deterministic": det,
        "rel_err_vs_fp64_same_tree_max": errs_max,
        "plain_fp64": {"value": plain, "ms_per_step": statistics.mean(pt), "n_max": N_MAX, "steps": args.fp64_steps},
        "speedup_vs_plain_fp64": value / plain,
        "learned_orders": {**info, "mean_p_qbx": float(qn.mean()), "mean_p_fmm_box": float(pn.mean())},
        "autotune": tuned, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("gpu", "reference"), default="gpu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-sub", type=int, default=None,
                    help="icosahedron face subdivision (default: the workload's; 20 = 8,000 elements)")
    ap.add_argument("--n-max", type=int, default=0, help="particles per leaf before a box splits (0: tuned value)")
    ap.add_argument("--mixed-form", choices=("fp32", "3xtf32"), default="3xtf32",
                    help="translation products of the learned mode: FP32 SIMT or split-TF32 tensor cores")
    ap.add_argument("--precision", choices=("fp64", "fp32", "3xtf32", "learned"), default="learned",
                    help="fp64: every stage FP64; fp32: List 2 M2L and List 3 far M2QBXL as FP32 products; "
                         "learned: fp32 with per-center / per-box orders from the trained network")
    ap.add_argument("--fp64-steps", type=int, default=5, help="timed steps of the plain FP64 comparison")
    ap.add_argument("--workload", choices=tuple(WORKLOADS) + ("batched",), default="star8k",
                    help="star8k (120k sources, default), star40k (607k), star79k (1.19M, random density, orders "
                         "8/16), or batched: many surfaces in one forest and graph")
    ap.add_argument("--batch", type=int, default=64, help="surfaces of the batched workload")
    ap.add_argument("--no-tune", action="store_true", help="batched: skip the leaf-size autotuner")
    ap.add_argument("--no-fp64-baseline", action="store_true")
    args = ap.parse_args()
    global P_QBX, P_FMM
    if args.workload in WORKLOADS:
        n_sub, _, _, (P_QBX, P_FMM), _ = WORKLOADS[args.workload]
        if args.n_sub is None:
            args.n_sub = n_sub
    elif args.n_sub is None:
        args.n_sub = 20
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
