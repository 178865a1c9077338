"""Failure handling of the tensor-core pipelines without a GPU fault.

A probe makes one wait of each tensor-core kernel run out on a barrier that nothing arrives on (with a
short limit); the kernel drains the copies and products it has issued, frees its tensor memory and
returns, and qbx_eval reports QBX_ERR_TIMEOUT.  The next evaluation with the default settings is
correct (bitwise equal to one taken before), so the context stays usable.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cu(a, dt=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dt is None else t.to(dt)).cuda()


def test_a_wait_that_runs_out_returns_timeout_and_the_next_evaluation_is_correct(star_small):
    import paper_1805_06106_gb300 as G
    from synth import greens_density

    s = star_small
    T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(s.tgt_xyz), n_max=16, t_f=0.9)
    L = G.qbx_build_lists(T)
    u, dudn = greens_density(s)
    args = (_cu(s.src_w), _cu(dudn), _cu(-u), _cu(s.src_n), _cu(s.tgt_ctr, torch.int32))
    ref = G.qbx_eval(T, L, *args, 7, 15, precision=G.QBX_M2L_3XTF32).clone()
    # first pipeline step of every block, then a step in the middle (products already issued)
    for step in (0, 3):
        G.qbx_lists_set_wait(L, 20000, step)
        with pytest.raises(G.QbxError) as e:
            G.qbx_eval(T, L, *args, 7, 15, precision=G.QBX_M2L_3XTF32)
        assert e.value.code == -5, str(e.value)
        G.qbx_lists_set_wait(L, 0, -1)
        again = G.qbx_eval(T, L, *args, 7, 15, precision=G.QBX_M2L_3XTF32)
        torch.cuda.synchronize()
        assert torch.equal(again, ref)
    # a short but sufficient limit on real waits changes nothing
    G.qbx_lists_set_wait(L, 1 << 26, -1)
    assert torch.equal(G.qbx_eval(T, L, *args, 7, 15, precision=G.QBX_M2L_3XTF32), ref)
    G.qbx_lists_set_wait(L, 0, -1)
    with pytest.raises(G.QbxError):
        G.qbx_lists_set_wait(L, -1, -1)
