"""Mixed-precision List 2 M2L and List 3 far M2QBXL against the FP64 oracle (<= 1e-6).

Two forms: FP32 SIMT products (QBX_M2L_FP32) and split-TF32 tensor-core products with FP32
accumulation (QBX_M2L_3XTF32).  The orders cover both tensor-core operand shapes (one and two
N blocks of the List 2 accumulator) and both register layouts of the harmonic generator."""
import numpy as np
import pytest

import oracle as O
from synth import greens_density, real_ylm

from conftest import rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6


def _cu(a, dt=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dt is None else t.to(dt)).cuda()


def _run(s, sigma, mu, t, tc, q, p, n_max, precision):
    import paper_1805_06106_gb300 as G

    T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(t), n_max=n_max, t_f=0.9)
    L = G.qbx_build_lists(T)
    args = (_cu(s.src_w), None if sigma is None else _cu(sigma), None if mu is None else _cu(mu), _cu(s.src_n),
            _cu(tc, torch.int32), q, p)
    fp64 = G.qbx_eval(T, L, *args).cpu().numpy()
    mixed = G.qbx_eval(T, L, *args, precision=precision).cpu().numpy()
    mixed2 = G.qbx_eval(T, L, *args, precision=precision).cpu().numpy()
    return fp64, mixed, mixed2


@pytest.mark.parametrize("form", ["fp32", "3xtf32"])
@pytest.mark.parametrize("q,p,n_max", [(5, 10, 16), (7, 15, 32), (8, 16, 64)])
def test_mixed_m2l_star_with_point_targets(star_small, q, p, n_max, form):
    import paper_1805_06106_gb300 as G

    prec = {"fp32": G.QBX_M2L_FP32, "3xtf32": G.QBX_M2L_3XTF32}[form]
    s = star_small
    u, dudn = greens_density(s)
    rng = np.random.default_rng(2)
    vol = rng.uniform(-2.0, 2.0, size=(3, 300))
    t = np.concatenate([s.tgt_xyz, vol], axis=1)
    tc = np.concatenate([s.tgt_ctr, -np.ones(300, np.int32)]).astype(np.int32)
    fp64, mixed, mixed2 = _run(s, dudn, -u, t, tc, q, p, n_max, prec)
    To = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, t, n_max=n_max, t_f=0.9)
    ref = O.fmm_eval(To, O.build_lists(To), s.src_xyz, s.src_w, dudn, -u, s.src_n, s.ctr_xyz, t, tc, q, p)
    assert rel_linf(fp64, ref) <= 1e-10
    err = rel_linf(mixed, ref)
    assert err <= TOL_MIXED, err
    assert err > 1e-14  # the FP32 path ran: its rounding is visible
    assert np.array_equal(mixed, mixed2)  # deterministic


@pytest.mark.parametrize("form", ["fp32", "3xtf32"])
def test_mixed_m2l_sphere_single_layer(sphere320, form):
    import paper_1805_06106_gb300 as G

    s = sphere320
    sig = real_ylm(2, 1, s.src_xyz)
    prec = {"fp32": G.QBX_M2L_FP32, "3xtf32": G.QBX_M2L_3XTF32}[form]
    fp64, mixed, _ = _run(s, sig, None, s.tgt_xyz, s.tgt_ctr, 5, 10, 16, prec)
    assert rel_linf(mixed, fp64) <= TOL_MIXED
