"""GPU parity of the modeled cost counts, the sweep labels and the prediction-to-order map
against the CPU oracle (integers: bit for bit), through the C ABI."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cu(a, dt=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dt is None else t.to(dt)).cuda()


def _pair(s, n_max, tgt=None):
    import paper_1805_06106_gb300 as G

    t = s.tgt_xyz if tgt is None else tgt
    T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(t), n_max=n_max, t_f=0.9)
    To = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, t, n_max=n_max, t_f=0.9)
    return T, G.qbx_build_lists(T), To, O.build_lists(To)


@pytest.mark.parametrize("n_max,orders", [(8, (5, 10)), (32, (7, 15)), (64, (8, 16))])
def test_lists_cost_matches_oracle(star_small, n_max, orders):
    import paper_1805_06106_gb300 as G

    T, L, To, Lo = _pair(star_small, n_max)
    q, p = orders
    got = G.qbx_lists_cost(L, q, p)
    assert got["count"] == O.lists_counts(To, Lo)
    want = O.lists_cost(To, Lo, q, p)
    for k in O.LIST_NAMES:
        assert got["ops"][k] == want[k], k
    assert got["stages"] == want["stages"] and got["total"] == want["total"]


def test_lists_cost_of_a_deeper_tree(sphere320):
    import paper_1805_06106_gb300 as G

    T, L, To, Lo = _pair(sphere320, 16)
    assert G.qbx_lists_cost(L, 5, 10)["count"] == O.lists_counts(To, Lo)


def test_order_labels_match_oracle():
    import paper_1805_06106_gb300 as G

    rng = np.random.default_rng(5)
    K, n = 9, 5000
    orders = [4, 6, 8, 10, 12, 14, 16, 18, 20]
    ref = rng.normal(size=n)
    # errors that shrink with the order plus occasional late bumps, NaN and inf columns
    vals = ref[None, :] + rng.normal(size=(K, n)) * np.exp(-1.3 * np.arange(K))[:, None]
    vals[K - 1] = ref
    bump = rng.random((K - 1, n)) < 0.03
    vals[:-1][bump] += 1e-3
    vals[2, :50] = np.nan
    vals[5, 50:80] = np.inf
    for tol in (1e-6, 1e-3, 0.0):
        got = G.qbx_order_labels(_cu(vals), orders, tol).cpu().numpy().astype(np.int32)
        assert np.array_equal(got, O.order_labels(vals, orders, tol)), tol


def test_orders_from_predictions_match_oracle(star_small):
    import paper_1805_06106_gb300 as G

    s = star_small
    rng = np.random.default_rng(6)
    vol = rng.uniform(-1.5, 1.5, size=(3, 40))
    t = np.concatenate([s.tgt_xyz, vol], axis=1)
    tc = np.concatenate([s.tgt_ctr, -np.ones(40, np.int32)]).astype(np.int32)
    T, L, To, Lo = _pair(s, 16, tgt=t)
    pred = np.stack([rng.uniform(-3, 15, s.n_ctr), rng.uniform(-3, 24, s.n_ctr)], 1).astype(np.float32)
    pred[::97] = np.nan
    pred[5] = [7.5, 9.0]  # exact sums: ceil(7.5 + 0.5) = 8, ceil(9 + 1) = 10
    for mq, mp, lo_q, hi_q, lo_p, hi_p, pdef, with_pts in ((0.5, 1.0, 2, 12, 4, 20, 16, True),
                                                            (0.0, 0.0, 0, 16, 0, 20, 7, False),
                                                            (2.25, 3.5, 3, 9, 5, 15, 15, True)):
        qc, pb = G.qbx_orders_from_mlp(T, L, _cu(pred), mq, mp, lo_q, hi_q, lo_p, hi_p, pdef,
                                       tgt_ctr=_cu(tc) if with_pts else None)
        q_o, p_o = O.orders_from_pred(To, pred, mq, mp, lo_q, hi_q, lo_p, hi_p, pdef, tgt_ctr=tc if with_pts else None)
        assert np.array_equal(qc.cpu().numpy().astype(np.int32), q_o)
        assert np.array_equal(pb.cpu().numpy().astype(np.int32), p_o)


def test_orders_fallback_matches_oracle(star_small):
    import paper_1805_06106_gb300 as G

    s = star_small
    rng = np.random.default_rng(9)
    vol = rng.uniform(-1.5, 1.5, size=(3, 40))
    t = np.concatenate([s.tgt_xyz, vol], axis=1)
    tc = np.concatenate([s.tgt_ctr, -np.ones(40, np.int32)]).astype(np.int32)
    T, L, To, Lo = _pair(s, 16, tgt=t)
    nt = t.shape[1]
    judge = rng.normal(size=nt)
    res = judge + rng.normal(size=nt) * 1e-6
    res[rng.choice(nt, 20, replace=False)] = np.nan
    q0 = rng.integers(2, 9, s.n_ctr).astype(np.int8)
    p0 = rng.integers(4, 17, T.n_boxes).astype(np.int8)
    qg, pg = _cu(q0), _cu(p0)
    n = G.qbx_orders_fallback(T, _cu(res), _cu(judge), _cu(tc), 2e-6, 8, 16, qg, pg)
    qo, po = q0.astype(np.int32), p0.astype(np.int32)
    no = O.orders_fallback(To, res, judge, tc, 2e-6, 8, 16, qo, po)
    assert n == no and n > 20
    assert np.array_equal(qg.cpu().numpy().astype(np.int32), qo)
    assert np.array_equal(pg.cpu().numpy().astype(np.int32), po)
