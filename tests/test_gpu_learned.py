"""Learned expansion orders: network kernels against the CPU oracle, labels, and the fixed-order acceptance check.

* The gradient of the training loss computed by the library's backward kernel equals the
  oracle's FP64 chain-rule gradient (FP32 tolerance).
* Training with the library's Adam kernel reduces the loss and is deterministic.
* The feature kernel equals the oracle's features (FP32 tolerance).
* On a surface held out of training, the orders the network picks give a result within
  1e-6 (normwise) of the fixed-order run that checks it, with no more work than that run (the
  per-box orders set the order of each box's local expansion); the work ratios are printed.
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cu(a, dt=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dt is None else t.to(dt)).cuda()


def test_backward_kernel_matches_oracle_gradient():
    import paper_1805_06106_gb300 as G

    rng = np.random.default_rng(0)
    params = G.qbx_mlp_init(seed=7)
    x = rng.normal(size=(300, 4)).astype(np.float32)
    t = rng.normal(size=(300, 2)).astype(np.float32) * 3
    g, loss = G.qbx_mlp_loss_grad(params, _cu(x), _cu(t))
    g_ref, loss_ref = O.mlp_loss_grad(params.cpu().numpy(), x, t)
    g = g.cpu().numpy().astype(np.float64)
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    assert abs(loss - loss_ref) <= 1e-5 * abs(loss_ref)
    # the forward kernel agrees with the same network
    y = G.qbx_mlp_forward(params, _cu(x)).cpu().numpy()
    p = params.cpu().numpy().astype(np.float64)
    h1 = np.tanh(x @ p[:256].reshape(64, 4).T + p[256:320])
    h2 = np.tanh(h1 @ p[320:4416].reshape(64, 64).T + p[4416:4480])
    yr = h2 @ p[4480:4608].reshape(2, 64).T + p[4608:4610]
    assert np.abs(y - yr).max() <= 1e-5 * np.abs(yr).max()


def test_training_reduces_loss_deterministically():
    import paper_1805_06106_gb300 as G

    rng = np.random.default_rng(1)
    x = rng.uniform(-2, 2, size=(4000, 4)).astype(np.float32)
    t = np.stack([np.round(5 + 2 * np.tanh(x[:, 0])), 8 + 4 * np.sin(x[:, 1]) + x[:, 2]], 1).astype(np.float32)
    runs = []
    for _ in range(2):
        params = G.qbx_mlp_init(seed=3)
        m, v = torch.zeros_like(params), torch.zeros_like(params)
        l0 = G.qbx_mlp_loss_grad(params, _cu(x), _cu(t))[1]
        l1 = G.qbx_mlp_train(params, m, v, _cu(x), _cu(t), 600, 1, 3e-3)
        runs.append((l0, l1, params.cpu().numpy()))
    assert runs[0][1] < 0.05 * runs[0][0]
    assert np.array_equal(runs[0][2], runs[1][2])


@pytest.mark.parametrize("layer", ["single", "double", "zero"])
def test_center_features_match_oracle(star_small, layer):
    """The feature kernel against the oracle's definition, element by element at FP32 tolerance
    (both compute in FP64 and round to float; log2/log10 may differ in the last FP64 bits)."""
    import paper_1805_06106_gb300 as G
    from synth import greens_density, random_harmonic_density

    s = star_small
    u, dudn = greens_density(s)
    sig, mu = {"single": (random_harmonic_density(s, 10, 3), None), "double": (dudn, -u),
               "zero": (np.zeros(s.n_src), None)}[layer]
    T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(s.tgt_xyz), n_max=16, t_f=0.9)
    L = G.qbx_build_lists(T)
    f = G.qbx_center_features(T, L, _cu(s.src_w), _cu(sig), None if mu is None else _cu(mu),
                              _cu(s.src_n)).cpu().numpy()
    To = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, s.tgt_xyz, n_max=16, t_f=0.9)
    ref = O.center_features(To, O.build_lists(To), s.src_w, sig, mu, s.src_n, s.ctr_xyz, s.ctr_r)
    assert np.array_equal(f[:, 1], ref[:, 1])
    assert np.allclose(f, ref, rtol=2e-7, atol=1e-6)


def test_learned_orders_pass_the_fixed_order_check_on_a_held_out_surface():
    import paper_1805_06106_gb300 as G
    from paper_1805_06106_gb300 import learned
    from synth import greens_density, make_surface, random_harmonic_density, real_ylm, star_radius
    from synth.surfaces import STAR_Y63, STAR_Y84_Y52

    q_fix, p_fix, tol, n_max = 8, 16, 1e-6, 64
    train = []
    for n, shape, seed in ((3, None, 11), (3, STAR_Y63, 12), (4, None, 13), (4, STAR_Y63, 14)):
        s = make_surface(n) if shape is None else make_surface(n, star_radius(shape))
        if shape is None:
            train.append(learned.sweep_samples(s, real_ylm(2, 1, s.src_xyz), None, q_fix, p_fix, n_max, tol))
        else:
            u, dudn = greens_density(s)
            train.append(learned.sweep_samples(s, dudn, -u, q_fix, p_fix, n_max, tol))
        train.append(learned.sweep_samples(s, random_harmonic_density(s, 10, seed), None, q_fix, p_fix, n_max, tol))
    params, losses = learned.train(train, steps=1000)
    assert losses[-1] < losses[0]
    mq, mp = learned.calibrate(params, train)

    s = make_surface(4, star_radius(STAR_Y84_Y52))  # held out: other surface, other density
    sig = random_harmonic_density(s, 10, 4)
    T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(s.tgt_xyz), n_max=n_max)
    L = G.qbx_build_lists(T)
    args = (_cu(s.src_w), _cu(sig), None, _cu(s.src_n), _cu(s.tgt_ctr, torch.int32))
    qc, pb = learned.predict_orders(T, L, params, args[0], args[1], None, args[3], q_range=(2, q_fix),
                                    p_range=(4, p_fix), margin_q=mq, margin_p=mp, p_default=p_fix, tgt_ctr=args[4])
    fixed = G.qbx_eval(T, L, *args, q_fix, p_fix).cpu().numpy()
    mixed = G.qbx_eval(T, L, *args, q_fix, p_fix, p_qbx_per_ctr=qc, p_fmm_per_box=pb,
                       precision=G.QBX_M2L_FP32).cpu().numpy()
    err = float(np.abs(mixed - fixed).max() / np.abs(fixed).max())
    q, p = qc.cpu().numpy().astype(int), pb.cpu().numpy().astype(int)
    work_q = np.sum((q + 1) * (q + 2)) / (s.n_ctr * (q_fix + 1) * (q_fix + 2))
    # L2QBXL work per center scales with (p_b + 1)^2 of its box's local expansion
    ctr_box = T.export()["ctr_owner"].cpu().numpy()
    work_l2q = np.sum((p[ctr_box] + 1) ** 2) / (s.n_ctr * (p_fix + 1) ** 2)
    print(f"learned orders: margins {mq:.2f}/{mp:.2f}, error vs fixed {err:.2e}, QBX-order work {work_q:.3f}, "
          f"L2QBXL work {work_l2q:.3f} of fixed, mean local order {p.mean():.2f}")
    assert err <= tol
    assert work_q <= 1.0
    assert work_l2q <= 1.0
