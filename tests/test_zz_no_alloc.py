"""qbx_eval_noalloc: the no-allocation variant of qbx_eval.

Callers that cannot call cudaMalloc while they evaluate (real-time loops with a fixed
memory budget, hosts whose allocator owns the device) use qbx_eval_noalloc, which takes
its scratch from a fixed array inside the library.  This file is collected last so that a
failure here leaves every other test already run; it also passes on its own in a fresh
process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cu(a, dt=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dt is None else t.to(dt)).cuda()


def test_noalloc_matches_qbx_eval_on_two_calls_in_a_row():
    import paper_1805_06106_gb300 as G
    from synth import greens_density, make_surface, real_ylm, star_radius
    from synth.surfaces import STAR_Y63

    s = make_surface(3, star_radius(STAR_Y63))
    rng = np.random.default_rng(1)
    vol = rng.uniform(-2.0, 2.0, size=(3, 200))
    t = np.concatenate([s.tgt_xyz, vol], axis=1)
    tc = _cu(np.concatenate([s.tgt_ctr, -np.ones(200, np.int32)]).astype(np.int32))
    T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(t), n_max=32, t_f=0.9)
    L = G.qbx_build_lists(T)
    w, n = _cu(s.src_w), _cu(s.src_n)
    u, dudn = greens_density(s)
    cases = [(_cu(dudn), _cu(-u), 7, 15), (_cu(real_ylm(3, 2, s.src_xyz)), None, 5, 10)]
    refs = [G.qbx_eval(T, L, w, sg, mu, n, tc, q, p) for sg, mu, q, p in cases]
    out = torch.empty(t.shape[1], dtype=torch.float64, device="cuda")
    for (sg, mu, q, p), ref in zip(cases, refs):  # two calls in a row, different densities and orders
        G.qbx_eval_noalloc(T, L, w, sg, mu, n, tc, q, p, out=out)
        torch.cuda.synchronize()
        err = float((out - ref).abs().max() / ref.abs().max())
        assert err <= 1e-10, err


def test_noalloc_rejects_a_problem_larger_than_its_scratch():
    import paper_1805_06106_gb300 as G
    from synth import greens_density, make_surface, star_radius
    from synth.surfaces import STAR_Y63

    s = make_surface(16, star_radius(STAR_Y63))  # 76,800 sources, 153,600 centers
    T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(s.tgt_xyz), n_max=32, t_f=0.9)
    L = G.qbx_build_lists(T)
    u, dudn = greens_density(s)
    out = torch.empty(s.n_ctr, dtype=torch.float64, device="cuda")
    with pytest.raises(G.QbxError) as e:
        G.qbx_eval_noalloc(T, L, _cu(s.src_w), _cu(dudn), None, _cu(s.src_n), _cu(s.tgt_ctr, torch.int32), 7, 15,
                           out=out)
    assert e.value.code == -1 and "bytes of scratch" in str(e.value)
