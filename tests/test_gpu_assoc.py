"""GPU target association (Algorithm 3) against the oracle's area-query implementation: bit for bit
(center indices and flags), with and without the side preference, on points near the surface and in
the volume, and the product path that feeds the associated volume points to qbx_eval."""
import numpy as np
import pytest

import oracle as O
from synth import danger_radius, make_surface, near_surface_points, star_radius, volume_points
from synth.surfaces import STAR_Y63

from conftest import rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cu(a, dt=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dt is None else t.to(dt)).cuda()


@pytest.mark.parametrize("n,n_max,sides,eps", [(3, 8, True, 0.05), (3, 32, False, 0.05), (5, 16, True, 0.0),
                                               (5, 48, True, 0.2)])
def test_association_matches_oracle(n, n_max, sides, eps):
    import paper_1805_06106_gb300 as G

    s = make_surface(n, star_radius(STAR_Y63))
    t = np.concatenate([near_surface_points(s, 4000, seed=7), volume_points(2000, seed=8, box=1.8)], axis=1)
    T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(t), n_max=n_max, t_f=0.9)
    rd = danger_radius(s)
    tc, fl = G.qbx_assoc_targets(T, _cu(rd), _cu(s.src_n) if sides else None,
                                 _cu(s.ctr_side.astype(np.int8)) if sides else None, eps)
    To = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, t, n_max=n_max, t_f=0.9)
    tco, flo = O.assoc_targets(To, s.src_xyz, rd, s.src_n if sides else None, s.ctr_xyz, s.ctr_r,
                               s.ctr_side if sides else None, t, eps)
    assert np.array_equal(tc.cpu().numpy(), tco)
    assert np.array_equal(fl.cpu().numpy().astype(bool), flo)
    assert (tco >= 0).sum() > 1000 and (tco < 0).sum() > 500


def test_associated_volume_points_evaluate_like_the_oracle():
    """Volume points associated on the GPU, then evaluated with the on-surface targets: the potential
    equals the oracle's on the same association (1e-10), inside points carry u, outside ones 0
    (Green's formula with the FP64 path, to quadrature accuracy)."""
    import paper_1805_06106_gb300 as G
    from synth import greens_density

    s = make_surface(4, star_radius(STAR_Y63))
    vol = np.concatenate([near_surface_points(s, 300, seed=9), volume_points(300, seed=10, box=1.8)], axis=1)
    Ta = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(vol), n_max=32, t_f=0.9)
    vc, vf = G.qbx_assoc_targets(Ta, _cu(danger_radius(s)), _cu(s.src_n), _cu(s.ctr_side.astype(np.int8)), 0.05)
    vc = vc.cpu().numpy()
    t = np.concatenate([s.tgt_xyz, vol], axis=1)
    tc = np.concatenate([s.tgt_ctr, vc]).astype(np.int32)
    u, dudn = greens_density(s)
    T = G.qbx_build_tree(_cu(s.src_xyz), _cu(s.ctr_xyz), _cu(s.ctr_r), _cu(t), n_max=32, t_f=0.9)
    L = G.qbx_build_lists(T)
    pot = G.qbx_eval(T, L, _cu(s.src_w), _cu(dudn), _cu(-u), _cu(s.src_n), _cu(tc, torch.int32), 7, 15).cpu().numpy()
    To = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, t, n_max=32, t_f=0.9)
    ref = O.fmm_eval(To, O.build_lists(To), s.src_xyz, s.src_w, dudn, -u, s.src_n, s.ctr_xyz, t, tc, 7, 15)
    assert rel_linf(pot, ref) <= 1e-10
    assert (vc >= 0).sum() > 100
