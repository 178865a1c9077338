"""Batched problems (a forest of independent surfaces) and captured evaluations (CUDA graphs).

* A forest evaluates every problem exactly as its own tree would: the concatenated result equals
  the separate runs bit for bit (each center, box and list pair is computed by the same
  arithmetic in the same order), in FP64 and in the split-TF32 tensor-core mode.
* One problem of the forest against the FP64 oracle (<= 1e-10).
* A captured evaluation replays to the eager result bit for bit, also after the density arrays
  are overwritten in place.
"""
import numpy as np
import pytest

import oracle as O
from synth import greens_density, make_surface, random_harmonic_density, star_radius
from synth.surfaces import STAR_Y63

from conftest import rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cu(a, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()


def _problems():
    """Three surfaces of different sizes and shapes; the second one also has volume targets."""
    out = []
    specs = [(2, None, 7), (3, STAR_Y63, 8), (2, [(0.25, 4, 2)], 9)]
    for i, (n, terms, seed) in enumerate(specs):
        s = make_surface(n) if terms is None else make_surface(n, star_radius(terms))
        if i == 1:
            u, dudn = greens_density(s)
            sigma, mu = dudn, -u
            vol = np.random.default_rng(3).uniform(-1.8, 1.8, size=(3, 40))
            t = np.concatenate([s.tgt_xyz, vol], axis=1)
            tc = np.concatenate([s.tgt_ctr, -np.ones(40, np.int32)]).astype(np.int32)
        else:
            sigma, mu = random_harmonic_density(s, 6, seed), None
            t, tc = s.tgt_xyz, s.tgt_ctr
        out.append(dict(s=s, sigma=sigma, mu=mu, t=t, tc=tc))
    return out


def _concat(probs, key, axis=-1):
    return np.concatenate([p[key] for p in probs], axis=axis)


@pytest.mark.parametrize("form", ["fp64", "3xtf32"])
def test_forest_equals_separate_runs(form):
    import paper_1805_06106_gb300 as G

    prec = {"fp64": G.QBX_FP64, "3xtf32": G.QBX_M2L_3XTF32}[form]
    q, p, n_max = 6, 12, 24
    probs = _problems()
    trees, lists, sep = [], [], []
    for pr in probs:
        s = pr["s"]
        T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(pr["t"]), n_max=n_max, t_f=0.9)
        L = G.qbx_build_lists(T)
        mu = None if pr["mu"] is None else _cu(pr["mu"])
        pot = G.qbx_eval(T, L, _cu(s.src_w), _cu(pr["sigma"]), mu, _cu(s.src_n), _cu(pr["tc"], torch.int32), q, p,
                         precision=prec)
        trees.append(T)
        lists.append(L)
        sep.append(pot.cpu().numpy())
    F, FL = G.qbx_build_forest(trees, lists)
    off = F.offsets
    assert F.n_problems == 3
    assert off["src"][-1] == sum(pr["s"].n_src for pr in probs)
    assert off["ctr"][-1] == sum(pr["s"].n_ctr for pr in probs)
    # concatenated inputs; densities absent on a problem are zero there (mu exists on one problem)
    w = _concat([dict(x=pr["s"].src_w) for pr in probs], "x")
    sigma = _concat(probs, "sigma")
    mu = np.concatenate([pr["mu"] if pr["mu"] is not None else np.zeros(pr["s"].n_src) for pr in probs])
    nrm = np.concatenate([pr["s"].src_n for pr in probs], axis=1)
    tc = np.concatenate([np.where(pr["tc"] >= 0, pr["tc"] + off["ctr"][i], -1) for i, pr in enumerate(probs)])
    pot = G.qbx_eval(F, FL, _cu(w), _cu(sigma), _cu(mu), _cu(nrm), _cu(tc.astype(np.int32), torch.int32), q, p,
                     precision=prec).cpu().numpy()
    for i, pr in enumerate(probs):
        part = pot[off["tgt"][i]:off["tgt"][i + 1]]
        if pr["mu"] is None and form == "fp64":
            # a zero double layer adds exact zeros: still the same numbers
            assert rel_linf(part, sep[i]) <= 1e-15
        elif pr["mu"] is None:
            assert rel_linf(part, sep[i]) <= 1e-12
        else:
            assert np.array_equal(part, sep[i])
    if form == "fp64":
        pr = probs[1]
        s = pr["s"]
        To = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, pr["t"], n_max=n_max, t_f=0.9)
        ref = O.fmm_eval(To, O.build_lists(To), s.src_xyz, s.src_w, pr["sigma"], pr["mu"], s.src_n, s.ctr_xyz,
                         pr["t"], pr["tc"], q, p)
        assert rel_linf(pot[off["tgt"][1]:off["tgt"][2]], ref) <= 1e-10


@pytest.mark.parametrize("form", ["fp64", "3xtf32"])
def test_graph_replay_matches_eager(form):
    import paper_1805_06106_gb300 as G

    prec = {"fp64": G.QBX_FP64, "3xtf32": G.QBX_M2L_3XTF32}[form]
    s = make_surface(3, star_radius(STAR_Y63))
    u, dudn = greens_density(s)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(s.tgt_xyz), n_max=32, t_f=0.9)
        L = G.qbx_build_lists(T)
        w, sg, mu, nrm = _cu(s.src_w), _cu(dudn), _cu(-u), _cu(s.src_n)
        tc = _cu(s.tgt_ctr, torch.int32)
        out = torch.empty(s.n_ctr, dtype=torch.float64, device="cuda")
        graph = G.qbx_graph_create(T, L, w, sg, mu, nrm, tc, 7, 15, out, precision=prec)
        first = out.clone()
        eager = G.qbx_eval(T, L, w, sg, mu, nrm, tc, 7, 15, precision=prec)
        out.zero_()
        graph.launch()
        replay = out.clone()
        # new densities in the same arrays
        sg.copy_(_cu(random_harmonic_density(s, 8, 11)))
        mu.mul_(0.5)
        graph.launch()
        replay2 = out.clone()
        eager2 = G.qbx_eval(T, L, w, sg, mu, nrm, tc, 7, 15, precision=prec)
    torch.cuda.synchronize()
    assert torch.equal(first, eager)
    assert torch.equal(replay, eager)
    assert torch.equal(replay2, eager2)
    assert not torch.equal(replay2, replay)


def test_graph_needs_a_stream():
    import paper_1805_06106_gb300 as G

    s = make_surface(2)
    T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(s.tgt_xyz), n_max=32, t_f=0.9)
    L = G.qbx_build_lists(T)
    out = torch.empty(s.n_ctr, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(torch.cuda.default_stream()):
        with pytest.raises(G.QbxError):
            G.qbx_graph_create(T, L, _cu(s.src_w), _cu(np.ones(s.n_src)), None, None, _cu(s.tgt_ctr, torch.int32),
                               4, 8, out)
