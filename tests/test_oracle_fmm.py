"""Whole-method pins of the oracle (no GPU).

* Algorithm 4 converges to direct (unaccelerated) QBX geometrically in p_fmm
  (Theorem 1; factor (3/4) per order for t_f <= 0.848, 0.771 at t_f = 0.9).
* Closed form on the unit sphere: S[Y_n^m] = Y_n^m / (2n+1) on the surface,
  r^n Y_n^m / (2n+1) inside and Y_n^m / ((2n+1) r^(n+1)) outside.
* Green's formula (Section 6.1): for u harmonic inside, S(d_n u) - D(u) is u at
  interior limits and in the interior, 0 at exterior limits and outside, u/2 on
  average.  Gauss's law D[1] = -1 inside, 0 outside.

On-surface limits use sources from a 4x finer mesh of the same surface than the
centers (the oversampling of Section 3.1, stage-2 quadrature), so that the
quadrature error is far below the sizes of the mistakes these pins catch.
"""
import math

import numpy as np
import pytest

import oracle as O
from synth import greens_density, make_surface, real_ylm, star_radius
from synth.surfaces import STAR_Y63

from conftest import rel_linf

TF = 0.9


def _fmm(surf, sigma, mu, p_qbx, p_fmm, n_max=32, tgt_xyz=None, tgt_ctr=None, **kw):
    t = surf.tgt_xyz if tgt_xyz is None else tgt_xyz
    tc = surf.tgt_ctr if tgt_ctr is None else tgt_ctr
    T = O.build_tree(surf.src_xyz, surf.ctr_xyz, surf.ctr_r, t, n_max=n_max, t_f=TF)
    L = O.build_lists(T)
    return O.fmm_eval(T, L, surf.src_xyz, surf.src_w, sigma, mu, surf.src_n, surf.ctr_xyz, t, tc, p_qbx, p_fmm, **kw)


def test_fmm_converges_to_direct_qbx_single_layer(sphere80):
    s = sphere80
    sig = real_ylm(2, 1, s.src_xyz)
    ref = O.direct_eval(s.src_xyz, s.src_w, sig, None, s.src_n, s.ctr_xyz, s.tgt_xyz, s.tgt_ctr, 5)
    errs = {p: rel_linf(_fmm(s, sig, None, 5, p), ref) for p in (4, 8, 12)}
    assert errs[4] > errs[8] > errs[12]
    assert errs[12] <= errs[4] * 0.7711 ** 8
    assert errs[12] < 1e-5


def test_fmm_converges_to_direct_qbx_double_layer_with_point_targets(star_small):
    s = star_small
    u, dudn = greens_density(s)
    rng = np.random.default_rng(3)
    vol = rng.uniform(-1.5, 1.5, size=(3, 300))
    vol = vol[:, np.linalg.norm(vol, axis=0) > 1.45]  # clear of the surface: plain quadrature targets
    t = np.concatenate([s.tgt_xyz, vol], axis=1)
    tc = np.concatenate([s.tgt_ctr, -np.ones(vol.shape[1], np.int32)])
    # direct reference on a sample of the QBX targets and on every point target
    sub = np.concatenate([rng.choice(s.n_ctr, 300, replace=False), np.arange(s.n_ctr, t.shape[1])])
    ref = O.direct_eval(s.src_xyz, s.src_w, dudn, -u, s.src_n, s.ctr_xyz, t[:, sub], tc[sub], 5)
    e4 = rel_linf(_fmm(s, dudn, -u, 5, 4, tgt_xyz=t, tgt_ctr=tc)[sub], ref)
    e8 = rel_linf(_fmm(s, dudn, -u, 5, 8, tgt_xyz=t, tgt_ctr=tc)[sub], ref)
    assert e8 <= e4 * 0.7711 ** 4
    assert e8 < 5e-4


def test_per_box_and_per_center_orders(sphere80):
    s = sphere80
    sig = real_ylm(2, 1, s.src_xyz)
    T = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, s.tgt_xyz, n_max=32, t_f=TF)
    L = O.build_lists(T)
    args = (T, L, s.src_xyz, s.src_w, sig, None, s.src_n, s.ctr_xyz, s.tgt_xyz, s.tgt_ctr)
    fixed = O.fmm_eval(*args, 5, 8)
    same = O.fmm_eval(*args, 5, 8, p_qbx_ctr=np.full(s.n_ctr, 5, np.int8), p_fmm_box=np.full(T.n_boxes, 8, np.int8))
    assert np.array_equal(fixed, same)
    rng = np.random.default_rng(0)
    pb = rng.integers(8, 13, T.n_boxes).astype(np.int8)
    mixed = O.fmm_eval(*args, 5, 8, p_fmm_box=pb)
    ref = O.direct_eval(s.src_xyz, s.src_w, sig, None, s.src_n, s.ctr_xyz, s.tgt_xyz, s.tgt_ctr, 5)
    assert rel_linf(mixed, ref) < rel_linf(fixed, ref) * 1.5  # mixed orders >= 8 are no worse than order 8


def _oversampled(radius_fn, n_ctr, n_src, nsub=40, seed=0):
    sc = make_surface(n_ctr, radius_fn)
    ss = make_surface(n_src, radius_fn)
    rng = np.random.default_rng(seed)
    sub = rng.choice(sc.n_src, nsub, replace=False)
    cidx = np.concatenate([sub, sub + sc.n_src])  # exterior then interior center of the same nodes
    return sc, ss, sub, cidx


def test_sphere_closed_form_on_surface():
    sc, ss, sub, cidx = _oversampled(lambda x: np.ones(x.shape[1]), 2, 8)
    for n, m in ((2, 1), (3, -2)):
        sig = real_ylm(n, m, ss.src_xyz)
        pot = O.direct_eval(ss.src_xyz, ss.src_w, sig, None, ss.src_n, sc.ctr_xyz[:, cidx], sc.tgt_xyz[:, cidx],
                            np.arange(cidx.size, dtype=np.int32), 7)
        ex = real_ylm(n, m, sc.src_xyz[:, sub]) / (2 * n + 1)
        k = sub.size
        assert rel_linf(pot[:k], ex) < 2e-3 and rel_linf(pot[k:], ex) < 2e-3


@pytest.mark.parametrize("r", [0.4, 2.5])
def test_sphere_closed_form_off_surface(sphere320, r):
    s = sphere320
    rng = np.random.default_rng(1)
    d = rng.normal(size=(3, 50))
    d /= np.linalg.norm(d, axis=0)
    for n, m in ((2, 1), (4, 3)):
        sig = real_ylm(n, m, s.src_xyz)
        pot = O.direct_eval(s.src_xyz, s.src_w, sig, None, s.src_n, s.ctr_xyz[:, :1], d * r,
                            -np.ones(50, np.int32), 5)
        ex = real_ylm(n, m, d) / (2 * n + 1) * (r ** n if r < 1 else r ** (-n - 1))
        assert rel_linf(pot, ex) < 1e-4  # smooth quadrature on the degree-4 polygonal sphere


def test_greens_formula_on_surface():
    sc, ss, sub, cidx = _oversampled(star_radius(STAR_Y63), 3, 12)
    u, dudn = greens_density(ss)
    uc, _ = greens_density(sc)
    pot = O.direct_eval(ss.src_xyz, ss.src_w, dudn, -u, ss.src_n, sc.ctr_xyz[:, cidx], sc.tgt_xyz[:, cidx],
                        np.arange(cidx.size, dtype=np.int32), 5)
    k = sub.size
    umax = np.abs(uc).max()
    ext, inte, uu = pot[:k], pot[k:], uc[sub]
    assert np.abs(ext).max() / umax < 2e-4  # exterior limit 0
    assert np.abs(inte - uu).max() / umax < 1e-4  # interior limit u
    assert np.abs(0.5 * (ext + inte) - 0.5 * uu).max() / umax < 1e-4  # principal value u/2


def test_greens_formula_and_gauss_law_in_volume(star_small):
    s = star_small
    u, dudn = greens_density(s)
    rng = np.random.default_rng(5)
    inside = rng.normal(size=(3, 40))
    inside *= 0.5 * rng.uniform(0, 1, 40) / np.linalg.norm(inside, axis=0)
    outside = rng.normal(size=(3, 40))
    outside *= rng.uniform(2.0, 3.0, 40) / np.linalg.norm(outside, axis=0)
    t = np.concatenate([inside, outside], axis=1)
    tc = -np.ones(80, np.int32)
    pot = O.direct_eval(s.src_xyz, s.src_w, dudn, -u, s.src_n, s.ctr_xyz[:, :1], t, tc, 5)
    x0 = np.array([3.0, 1.0, 2.0])
    uin = 1.0 / np.linalg.norm(inside - x0[:, None], axis=0)
    # plain quadrature away from the surface; residual is the degree-4 geometry error
    assert rel_linf(pot[:40], uin) < 5e-5
    assert np.abs(pot[40:]).max() / np.abs(uin).max() < 5e-5
    gauss = O.direct_eval(s.src_xyz, s.src_w, None, np.ones(s.n_src), s.src_n, s.ctr_xyz[:, :1], t, tc, 5)
    assert np.abs(gauss[:40] + 1.0).max() < 5e-5 and np.abs(gauss[40:]).max() < 5e-5


def test_single_layer_kernel_normalisation():
    """A unit charge: the potential is exactly 1/(4 pi r) (eq. laplace-fs-green)."""
    s = np.array([[0.3], [-0.2], [0.1]])
    t = np.array([[1.3], [0.8], [-0.9]])
    pot = O.direct_eval(s, np.ones(1), np.ones(1), None, np.zeros((3, 1)), s, t, -np.ones(1, np.int32), 3)
    assert abs(pot[0] - 1 / (4 * math.pi * np.linalg.norm(t - s))) < 1e-17


def test_openmp_build_gives_the_serial_result(sphere80):
    """The all-cores build of the oracle (used only to time the CPU baseline) runs the same loops over
    independent boxes and centers, each result accumulated in the same order: bitwise equal."""
    from synth import greens_density

    s = sphere80
    u, dudn = greens_density(s)
    T = O.build_tree(s.src_xyz, s.ctr_xyz, s.ctr_r, s.tgt_xyz, n_max=8, t_f=0.9)
    L = O.build_lists(T)
    args = (T, L, s.src_xyz, s.src_w, dudn, -u, s.src_n, s.ctr_xyz, s.tgt_xyz, s.tgt_ctr, 5, 10)
    try:
        par = O.fmm_eval(*args, omp=True)
    except RuntimeError as e:
        pytest.skip(str(e))
    assert np.array_equal(O.fmm_eval(*args), par)
