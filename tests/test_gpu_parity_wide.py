"""GPU parity on the configurations the benchmark paths take, against the FP64 oracle.

* A mid-size surface (19,200 sources, 38,400 centers, trees of 7+ levels, several tensor-core tiles per
  List 2 offset): FP64 within 1e-10, both mixed forms within 1e-6.
* The largest orders the API allows: p_fmm = 20 (two accumulator blocks of the List 2 products) and
  p_qbx in {12, 16}.
* The non-default K-chunk hints of the tensor-core kernels.
* The combination the learned benchmark runs: per-center and per-box orders from the order network,
  checked by the fixed-order judge, split-TF32 translations, a forest of surfaces, replayed as a CUDA
  graph; each surface against the oracle with the same orders (1e-6) and against the fixed-order
  oracle result (1e-6).
The oracle runs its OpenMP build (bitwise equal to the serial one) to keep these cases short.
"""
import numpy as np
import pytest

import oracle as O
from synth import greens_density, make_surface, random_harmonic_density, star_radius
from synth.surfaces import STAR_Y63, STAR_Y84_Y52

from conftest import rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cu(a, dt=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dt is None else t.to(dt)).cuda()


def _omp():
    try:
        O.lib_omp()
        return True
    except RuntimeError:
        return False


def _oracle(s, sigma, mu, t, tc, q, p, n_max, qctr=None, pbox=None):
    To = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, t, n_max=n_max, t_f=0.9)
    return O.fmm_eval(To, O.build_lists(To), s.src_xyz, s.src_w, sigma, mu, s.src_n, s.ctr_xyz, t, tc, q, p,
                      p_qbx_ctr=qctr, p_fmm_box=pbox, omp=_omp())


def _gpu(s, sigma, mu, t, tc, q, p, n_max, precision, tiles=None, T=None, L=None):
    import paper_1805_06106_gb300 as G

    if T is None:
        T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(t), n_max=n_max, t_f=0.9)
        L = G.qbx_build_lists(T)
    if tiles is not None:
        G.qbx_lists_set_tiles(L, *tiles)
    out = G.qbx_eval(T, L, _cu(s.src_w), None if sigma is None else _cu(sigma), None if mu is None else _cu(mu),
                     _cu(s.src_n), _cu(tc, torch.int32), q, p, precision=precision)
    return out.cpu().numpy(), T, L


@pytest.fixture(scope="module")
def mid():
    s = make_surface(8, star_radius(STAR_Y63))  # 1,280 elements: 19,200 sources, 38,400 centers
    u, dudn = greens_density(s)
    vol = np.random.default_rng(11).uniform(-2.0, 2.0, size=(3, 500))
    t = np.concatenate([s.tgt_xyz, vol], axis=1)
    tc = np.concatenate([s.tgt_ctr, -np.ones(500, np.int32)]).astype(np.int32)
    ref = _oracle(s, dudn, -u, t, tc, 7, 15, 32)
    return dict(s=s, sigma=dudn, mu=-u, t=t, tc=tc, ref=ref)


def test_mid_size_surface_all_precisions(mid):
    import paper_1805_06106_gb300 as G

    m = mid
    fp64, T, L = _gpu(m["s"], m["sigma"], m["mu"], m["t"], m["tc"], 7, 15, 32, G.QBX_FP64)
    assert T.info.n_levels >= 7
    assert rel_linf(fp64, m["ref"]) <= 1e-10
    for prec in (G.QBX_M2L_FP32, G.QBX_M2L_3XTF32):
        mixed, _, _ = _gpu(m["s"], m["sigma"], m["mu"], m["t"], m["tc"], 7, 15, 32, prec, T=T, L=L)
        err = rel_linf(mixed, m["ref"])
        assert 1e-14 < err <= 1e-6, (prec, err)


@pytest.mark.parametrize("tiles", [(16, 48), (32, 64), (16, 16), (32, 128)])
def test_tensor_core_chunk_hints(mid, tiles):
    import paper_1805_06106_gb300 as G

    m = mid
    mixed, _, _ = _gpu(m["s"], m["sigma"], m["mu"], m["t"], m["tc"], 7, 15, 32, G.QBX_M2L_3XTF32, tiles=tiles)
    assert rel_linf(mixed, m["ref"]) <= 1e-6


@pytest.mark.parametrize("q,p", [(12, 20), (16, 20), (16, 16)])
def test_highest_orders(star_small, q, p):
    import paper_1805_06106_gb300 as G

    s = star_small
    sig = random_harmonic_density(s, 10, 5)
    ref = _oracle(s, sig, None, s.tgt_xyz, s.tgt_ctr, q, p, 32)
    fp64, T, L = _gpu(s, sig, None, s.tgt_xyz, s.tgt_ctr, q, p, 32, G.QBX_FP64)
    assert rel_linf(fp64, ref) <= 1e-10
    mixed, _, _ = _gpu(s, sig, None, s.tgt_xyz, s.tgt_ctr, q, p, 32, G.QBX_M2L_3XTF32, T=T, L=L)
    assert rel_linf(mixed, ref) <= 1e-6


def test_learned_split_tf32_forest_graph_against_oracle():
    """Orders from a network trained by the library's kernels on order sweeps of two small surfaces,
    applied to a forest of three other surfaces evaluated with split-TF32 translations and replayed
    as a CUDA graph."""
    import paper_1805_06106_gb300 as G
    from paper_1805_06106_gb300 import learned

    q_fix, p_fix, n_max, tol = 8, 16, 32, 1e-6
    train = []
    for n, shape, seed in ((3, STAR_Y63, 21), (3, None, 22)):
        s = make_surface(n) if shape is None else make_surface(n, star_radius(shape))
        train.append(learned.sweep_samples(s, random_harmonic_density(s, 10, seed), None, q_fix, p_fix, n_max, tol))
    model = learned.fit(train, steps=300)
    specs = [(2, STAR_Y84_Y52, 31), (3, [(0.2, 4, 2)], 32), (2, None, 33)]
    surfs = [make_surface(n) if sh is None else make_surface(n, star_radius(sh)) for n, sh, _ in specs]
    dens = [random_harmonic_density(s, 10, seed) for s, (_, _, seed) in zip(surfs, specs)]
    trees, lists = [], []
    for s in surfs:
        T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(s.tgt_xyz), n_max=n_max, t_f=0.9)
        trees.append(T)
        lists.append(G.qbx_build_lists(T))
    F, FL = G.qbx_build_forest(trees, lists)
    off = F.offsets
    w = _cu(np.concatenate([s.src_w for s in surfs]))
    sg = _cu(np.concatenate(dens))
    nrm = _cu(np.concatenate([s.src_n for s in surfs], axis=1))
    tc = _cu(np.concatenate([s.tgt_ctr + off["ctr"][i] for i, s in enumerate(surfs)]).astype(np.int32), torch.int32)
    qc, pb = learned.predict_orders(F, FL, model, w, sg, None, nrm, tgt_ctr=tc, q_range=(2, q_fix),
                                    p_range=(4, p_fix), p_default=p_fix)
    # the fixed-order FP64 judge raises the orders of the targets the network's orders miss
    qc, pb, info = learned.judge_and_fallback(F, FL, (w, sg, None, nrm, tc), q_fix, p_fix, qc, pb, 0.9 * tol,
                                              G.QBX_M2L_3XTF32)
    assert info["err_after"] <= 0.9 * tol
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        pot = torch.empty(int(F.info.n_tgt), dtype=torch.float64, device="cuda")
        g = G.qbx_graph_create(F, FL, w, sg, None, nrm, tc, q_fix, p_fix, pot, p_qbx_per_ctr=qc, p_fmm_per_box=pb,
                               precision=G.QBX_M2L_3XTF32)
        eager = pot.clone()
        pot.zero_()
        g.launch()
    torch.cuda.synchronize()
    res = pot.cpu().numpy()
    assert np.array_equal(res, eager.cpu().numpy())
    qn, pn = qc.cpu().numpy(), pb.cpu().numpy()
    for i, s in enumerate(surfs):
        sl = slice(off["tgt"][i], off["tgt"][i + 1])
        qi = qn[off["ctr"][i]:off["ctr"][i + 1]]
        pi = pn[off["boxes"][i]:off["boxes"][i + 1]]
        same = _oracle(s, dens[i], None, s.tgt_xyz, s.tgt_ctr, q_fix, p_fix, n_max, qctr=qi, pbox=pi)
        fixed = _oracle(s, dens[i], None, s.tgt_xyz, s.tgt_ctr, q_fix, p_fix, n_max)
        assert rel_linf(res[sl], same) <= 1e-6
        assert rel_linf(res[sl], fixed) <= tol
