"""Synthetic curved-triangle surfaces shaped like the paper's test geometries.

Recipe (Section 6 test geometries; Section 2.3 discretization; Section 3.2
expansion radii; eq. (expansion-centers)):

* The regular icosahedron is split into 20 n^2 flat sub-triangles.  On each one,
  15 equispaced barycentric points (degree 4) are projected radially onto the
  surface ``x = r(x_hat) x_hat``; they define a degree-4 Lagrange element map
  Psi_k from the unit right triangle (Section 2.3, element mappings).
* Sources are the 15 nodes of a conical-product (Stroud) rule on each element:
  5 Gauss-Jacobi(alpha=1, beta=0) points in the collapsed direction times
  3 Gauss-Legendre points, exact for total degree 5.  Each source weight is the
  rule weight times the area element |d1 Psi x d2 Psi| (Section 2.3).
* The resolution measure eta_k (eq. stretch-factor) is the maximum over the
  element's 15 quadrature and 15 geometry nodes of twice the largest singular
  value of the map's Jacobian composed with the map from the bi-unit
  equilateral triangle; the expansion radius is r_k = eta_k / 2
  (eq. expansion-radii).
* Two centers per node, x_i + r n_i (exterior) and x_i - r n_i (interior)
  (eq. expansion-centers).  One on-surface target per center at x_i.

Everything is float64 and deterministic for a given argument set.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# spherical harmonics used only to shape surfaces and densities
# --------------------------------------------------------------------------


def _legendre_nocs(n: int, m: int, x: np.ndarray) -> np.ndarray:
    """Associated Legendre function P_n^m(x), m >= 0, without the (-1)^m phase."""
    from scipy.special import lpmv

    return ((-1.0) ** m) * lpmv(m, n, x)


def real_ylm(n: int, m: int, xyz: np.ndarray) -> np.ndarray:
    """Real basis harmonic of direction xyz (3, N): Re Y_n^m for m >= 0, Im Y_n^|m| for m < 0.

    Y_n^m uses the normalisation of eq. (spherical-harmonics):
    sqrt((2n+1)/(4 pi) (n-|m|)!/(n+|m|)!) P_n^|m|(cos theta) e^{i m phi}.
    """
    x, y, z = xyz
    r = np.sqrt(x * x + y * y + z * z)
    ct = np.clip(z / r, -1.0, 1.0)
    ph = np.arctan2(y, x)
    am = abs(m)
    norm = math.sqrt((2 * n + 1) / (4 * math.pi) * math.factorial(n - am) / math.factorial(n + am))
    base = norm * _legendre_nocs(n, am, ct)
    return base * (np.cos(am * ph) if m >= 0 else np.sin(am * ph))


def sphere_radius(xhat: np.ndarray) -> np.ndarray:
    return np.ones(xhat.shape[1])


def star_radius(terms):
    """r(x_hat) = 1 + sum_k a_k Re Y_{n_k}^{m_k}(x_hat); terms = [(a, n, m), ...]."""

    def radius(xhat: np.ndarray) -> np.ndarray:
        r = np.ones(xhat.shape[1])
        for a, n, m in terms:
            r = r + a * real_ylm(n, m, xhat)
        return r

    return radius


def urchin_radius(k: int):
    """The 'urchin' gamma_k of Section 6.1 (eq. urchin-warping): r_k = 0.2 + (Re Y_k^{floor(k/2)} - m_k) /
    (M_k - m_k), M_k and m_k the largest and smallest value of Re Y_k^{floor(k/2)} on the sphere.  Re Y
    is N P_k^m(cos theta) cos(m phi), so for m > 0 the extremes are +- N max |P_k^m| (cos(m phi) = +-1),
    found by dense sampling in theta refined by golden-section search; for m = 0 they are the extremes
    of N P_k(cos theta)."""
    m = k // 2
    norm = math.sqrt((2 * k + 1) / (4 * math.pi) * math.factorial(k - m) / math.factorial(k + m))

    def f(t):
        return norm * _legendre_nocs(k, m, np.cos(np.atleast_1d(t)))

    def extreme(sign):
        t = np.linspace(0.0, math.pi, 20001)
        v = sign * f(t)
        i = int(np.argmax(v))
        lo, hi = t[max(i - 1, 0)], t[min(i + 1, len(t) - 1)]
        g = (math.sqrt(5.0) - 1.0) / 2.0
        for _ in range(200):  # golden-section refinement of the sampled maximum
            a_, b_ = hi - g * (hi - lo), lo + g * (hi - lo)
            if sign * f(a_)[0] > sign * f(b_)[0]:
                hi = b_
            else:
                lo = a_
        return float(sign * max(sign * f(lo)[0], sign * f(hi)[0], v[i]))

    if m > 0:
        M = max(extreme(1.0), -extreme(-1.0))
        mk = -M
    else:
        M, mk = extreme(1.0), extreme(-1.0)

    def radius(xhat: np.ndarray) -> np.ndarray:
        return 0.2 + (real_ylm(k, m, xhat) - mk) / (M - mk)

    radius.extremes = (mk, M)
    return radius


# --------------------------------------------------------------------------
# reference-triangle quadrature
# --------------------------------------------------------------------------


def _golub_welsch_jacobi(npts: int, alpha: float, beta: float):
    """Gauss-Jacobi nodes/weights on [-1, 1] for weight (1-t)^alpha (1+t)^beta (Golub-Welsch)."""
    ab = alpha + beta
    a = np.empty(npts)
    b = np.empty(max(npts - 1, 0))
    for k in range(npts):
        den = (2 * k + ab) * (2 * k + ab + 2)
        a[k] = (beta * beta - alpha * alpha) / den if den != 0 else (beta - alpha) / (ab + 2)
    for k in range(1, npts):
        num = 4.0 * k * (k + alpha) * (k + beta) * (k + ab)
        den = (2 * k + ab) ** 2 * (2 * k + ab + 1) * (2 * k + ab - 1)
        b[k - 1] = math.sqrt(num / den)
    jac = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    t, v = np.linalg.eigh(jac)
    mu0 = 2.0 ** (ab + 1) * math.gamma(alpha + 1) * math.gamma(beta + 1) / math.gamma(ab + 2)
    w = mu0 * v[0, :] ** 2
    return t, w


def triangle_rule():
    """15-node conical-product rule on the unit right triangle {u, v >= 0, u + v <= 1}.

    Duffy collapse u = xi, v = (1 - xi) eta with Jacobian (1 - xi): 5-point
    Gauss-Jacobi(1, 0) in xi and 3-point Gauss-Legendre in eta.  Exact for
    every monomial u^a v^b with b <= 5 and a + b <= 9 (so total degree 5).
    Returns (u, v, w) with sum(w) = 1/2.
    """
    tj, wj = _golub_welsch_jacobi(5, 1.0, 0.0)
    xi = 0.5 * (tj + 1.0)
    wxi = wj / 4.0
    tl, wl = np.polynomial.legendre.leggauss(3)
    eta = 0.5 * (tl + 1.0)
    weta = 0.5 * wl
    u = np.repeat(xi, 3)
    v = (1.0 - u) * np.tile(eta, 5)
    w = np.repeat(wxi, 3) * np.tile(weta, 5)
    return u, v, w


# degree-4 Lagrange element on the unit right triangle
_GEO_IJ = [(i, j) for j in range(5) for i in range(5 - j)]  # 15 nodes (u, v) = (i/4, j/4)
_MONO = [(a, b) for a in range(5) for b in range(5 - a)]


def _lagrange_coeffs():
    pts = np.array([(i / 4.0, j / 4.0) for i, j in _GEO_IJ])
    vander = np.array([[p[0] ** a * p[1] ** b for a, b in _MONO] for p in pts])
    return np.linalg.inv(vander)  # column k: monomial coefficients of basis k


_LAG = _lagrange_coeffs()


def _lagrange_eval(u: np.ndarray, v: np.ndarray):
    """Values and (d/du, d/dv) of the 15 degree-4 Lagrange basis functions at (u, v)."""
    mono = np.stack([u ** a * v ** b for a, b in _MONO], axis=-1)
    du = np.stack([a * u ** max(a - 1, 0) * v ** b if a > 0 else 0 * u for a, b in _MONO], axis=-1)
    dv = np.stack([b * u ** a * v ** max(b - 1, 0) if b > 0 else 0 * u for a, b in _MONO], axis=-1)
    return mono @ _LAG, du @ _LAG, dv @ _LAG


def _lagrange_eval2(u: np.ndarray, v: np.ndarray):
    """Second derivatives (d2/du2, d2/dudv, d2/dv2) of the 15 degree-4 Lagrange basis functions."""
    def mono(a, b, da, db):
        c = 1.0
        for k in range(da):
            c *= a - k
        for k in range(db):
            c *= b - k
        if c == 0.0:
            return 0 * u
        return c * u ** (a - da) * v ** (b - db)
    uu = np.stack([mono(a, b, 2, 0) for a, b in _MONO], axis=-1)
    uv = np.stack([mono(a, b, 1, 1) for a, b in _MONO], axis=-1)
    vv = np.stack([mono(a, b, 0, 2) for a, b in _MONO], axis=-1)
    return uu @ _LAG, uv @ _LAG, vv @ _LAG


def _icosahedron():
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    verts = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            verts += [(0.0, s1, s2 * phi), (s1, s2 * phi, 0.0), (s2 * phi, 0.0, s1)]
    verts = np.array(verts)
    verts /= np.linalg.norm(verts, axis=1)[:, None]
    # faces: all triples of mutually nearest vertices (edge length is the minimum distance)
    d = np.linalg.norm(verts[:, None, :] - verts[None, :, :], axis=-1)
    emin = np.min(d[d > 1e-9])
    adj = np.abs(d - emin) < 1e-9
    faces = []
    for a in range(12):
        for b in range(a + 1, 12):
            for c in range(b + 1, 12):
                if adj[a, b] and adj[b, c] and adj[a, c]:
                    A, B, C = verts[a], verts[b], verts[c]
                    if np.dot(np.cross(B - A, C - A), A + B + C) < 0:
                        b2, c2 = c, b
                    else:
                        b2, c2 = b, c
                    faces.append((a, b2, c2))
    assert len(faces) == 20
    return verts, np.array(faces)


def conical_rule(n: int):
    """Conical-product rule on the unit right triangle with n x n nodes (n-point Gauss-Jacobi(1, 0) in
    the collapsed direction, n-point Gauss-Legendre along it), exact to total degree 2n - 1."""
    tj, wj = _golub_welsch_jacobi(n, 1.0, 0.0)
    xi, wxi = 0.5 * (tj + 1.0), wj / 4.0
    tl, wl = np.polynomial.legendre.leggauss(n)
    eta, weta = 0.5 * (tl + 1.0), 0.5 * wl
    u = np.repeat(xi, n)
    return u, (1.0 - u) * np.tile(eta, n), np.repeat(wxi, n) * np.tile(weta, n)


def _orthonormal_by_degree():
    """Values at a degree-9 rule of an L2-orthonormal basis of P_4 on the unit triangle, ordered by
    total degree (Gram-Schmidt of the monomials in the order of _MONO sorted by degree), with each
    function's degree: the hierarchical split P_d = P_{d-1} + (its orthogonal complement) that a
    Dubiner (Koornwinder) basis also has."""
    u, v, w = conical_rule(5)
    order = sorted(range(len(_MONO)), key=lambda i: (sum(_MONO[i]), _MONO[i][1]))
    vals, degs = [], []
    for i in order:
        a, b = _MONO[i]
        q = u ** a * v ** b
        for p in vals:  # twice, for stability
            q = q - np.sum(w * q * p) * p
        for p in vals:
            q = q - np.sum(w * q * p) * p
        q = q / math.sqrt(np.sum(w * q * q))
        vals.append(q)
        degs.append(a + b)
    return u, v, w, np.array(vals), np.array(degs)


def map_tail(flat: np.ndarray, radius_fn=sphere_radius) -> np.ndarray:
    """Per element, the l2 norm of the coefficients of total degree 3 and 4 (the two highest) of the
    degree-4 element map in an orthonormal basis of the triangle, relative to the norm of all of them
    (the resolution measure of the adaptive meshing of Section 6.1)."""
    return _tail_of_geometry(_element_geometry(flat, radius_fn, 1.0, (0.0, 0.0, 0.0)))


def _tail_of_geometry(geo: np.ndarray) -> np.ndarray:
    """map_tail of degree-4 element maps given by their 15 geometry nodes (K, 15, 3)."""
    u, v, w, B, deg = _orthonormal_by_degree()
    phi, _, _ = _lagrange_eval(u, v)
    x = np.einsum("qb,kbd->kqd", phi, geo)                    # the map at the rule's nodes
    c = np.einsum("jq,q,kqd->kjd", B, w, x)                   # coefficients per basis function
    hi = deg >= 3
    return np.sqrt(np.sum(c[:, hi] ** 2, axis=(1, 2)) / np.sum(c ** 2, axis=(1, 2)))


def adaptive_flat_mesh(radius_fn, tol: float = 1e-4, max_rounds: int = 12):
    """Mesh of the surface r(x_hat) refined where its degree-4 element maps are not resolved (Section
    6.1): start from the icosahedron's faces and bisect every element whose map_tail exceeds tol,
    re-evaluating the map on the children, until none does.  Returns (flat mesh, tails per round)."""
    flat = _flat_subtriangles(1)
    hist = []
    for _ in range(max_rounds):
        t = map_tail(flat, radius_fn)
        marks = t > tol
        hist.append(int(marks.sum()))
        if not marks.any():
            return flat, hist
        flat = bisect_flat(flat, marks)
    raise RuntimeError(f"adaptive meshing did not resolve the maps in {max_rounds} rounds: {hist}")


def flat_mesh(n_sub: int) -> np.ndarray:
    """The uniform starting mesh: (K, 3, 3) flat sub-triangles of the icosahedron's faces."""
    return _flat_subtriangles(n_sub)


def bisect_flat(flat: np.ndarray, marks: np.ndarray) -> np.ndarray:
    """Mesh after bisection of the marked elements (Section 3.1): each marked flat triangle
    (A, B, C) is replaced by its four midpoint children, orientation kept; unmarked elements keep
    their index order, the children follow them in order of their parents."""
    marks = np.asarray(marks, bool)
    keep = flat[~marks]
    A, B, C = flat[marks, 0], flat[marks, 1], flat[marks, 2]
    ab, bc, ca = 0.5 * (A + B), 0.5 * (B + C), 0.5 * (C + A)
    kids = np.stack([np.stack([A, ab, ca], 1), np.stack([ab, B, bc], 1), np.stack([ca, bc, C], 1),
                     np.stack([ab, bc, ca], 1)], axis=1).reshape(-1, 3, 3)
    return np.concatenate([keep, kids], axis=0)


def _flat_subtriangles(n_sub: int) -> np.ndarray:
    """(K, 3, 3) flat sub-triangle vertices, outward-oriented, K = 20 n_sub^2."""
    verts, faces = _icosahedron()
    tris = []
    for a, b, c in faces:
        A, B, C = verts[a], verts[b], verts[c]

        def P(i, j):
            return A + (i / n_sub) * (B - A) + (j / n_sub) * (C - A)

        for j in range(n_sub):
            for i in range(n_sub - j):
                tris.append((P(i, j), P(i + 1, j), P(i, j + 1)))
                if i + j <= n_sub - 2:
                    tris.append((P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)))
    return np.array(tris)


# --------------------------------------------------------------------------
# surface assembly
# --------------------------------------------------------------------------


@dataclass
class Surface:
    """Discretised surface.  Arrays of points are SoA (3, N), float64."""

    n_elem: int
    src_xyz: np.ndarray  # (3, N_S) quadrature nodes
    src_w: np.ndarray  # (N_S,) rule weight x area element
    src_n: np.ndarray  # (3, N_S) outward unit normals
    src_elem: np.ndarray  # (N_S,) element index
    elem_eta: np.ndarray  # (K,) resolution measure eta_k
    ctr_xyz: np.ndarray  # (3, N_C) centers: [exterior (+) for all nodes, interior (-) for all nodes]
    ctr_r: np.ndarray  # (N_C,) expansion radius
    ctr_side: np.ndarray  # (N_C,) +1 exterior, -1 interior
    tgt_xyz: np.ndarray  # (3, N_T) on-surface targets, one per center
    tgt_ctr: np.ndarray  # (N_T,) int32 associated center
    radius_fn: object = field(repr=False, default=None)
    ctr_elem: np.ndarray = field(repr=False, default=None)     # (N_C,) element that spawned each center
    ctr_elem_eta: np.ndarray = field(repr=False, default=None)  # eta of the centers' elements (stage 1)
    interp: np.ndarray = field(repr=False, default=None)  # (sources, nodes) per element: node values -> sources

    @property
    def n_src(self) -> int:
        return self.src_xyz.shape[1]

    @property
    def n_ctr(self) -> int:
        return self.ctr_xyz.shape[1]


_AINV = np.array([[math.sqrt(3.0), -1.0], [0.0, 2.0]]) / (2.0 * math.sqrt(3.0))  # inverse of [[2,1],[0,sqrt3]]


def _stretch(du: np.ndarray, dv: np.ndarray) -> np.ndarray:
    """2 sigma_1(J A^{-1}) for Jacobian columns du, dv (..., 3) (eq. stretch-factor)."""
    c0 = du * _AINV[0, 0] + dv * _AINV[1, 0]
    c1 = du * _AINV[0, 1] + dv * _AINV[1, 1]
    g00 = np.sum(c0 * c0, -1)
    g11 = np.sum(c1 * c1, -1)
    g01 = np.sum(c0 * c1, -1)
    tr = g00 + g11
    det = g00 * g11 - g01 * g01
    lam = 0.5 * (tr + np.sqrt(np.maximum(tr * tr - 4.0 * det, 0.0)))
    return 2.0 * np.sqrt(lam)


def _upsampled_rule(f: int):
    """The 15-node rule on each of the f^2 congruent sub-triangles of the unit triangle (weights
    scaled by the area ratio 1/f^2): nodes of a finer source quadrature on the same element."""
    qu, qv, qw = triangle_rule()
    us, vs, ws = [], [], []
    for a in range(f):
        for b in range(f - a):
            # upright sub-triangle with corner (a, b)/f, and the inverted one above it
            corners = [((a, b), (a + 1, b), (a, b + 1))]
            if a + b < f - 1:
                corners.append(((a + 1, b + 1), (a, b + 1), (a + 1, b)))
            for (p0, p1, p2) in corners:
                A = np.array(p0, float) / f
                B = np.array(p1, float) / f
                C = np.array(p2, float) / f
                us.append(A[0] + qu * (B[0] - A[0]) + qv * (C[0] - A[0]))
                vs.append(A[1] + qu * (B[1] - A[1]) + qv * (C[1] - A[1]))
                ws.append(qw / (f * f))
    return np.concatenate(us), np.concatenate(vs), np.concatenate(ws)


def make_surface(n_sub: int, radius_fn=sphere_radius, scale: float = 1.0, offset=(0.0, 0.0, 0.0),
                 upsample: int = 1) -> Surface:
    """Curved triangles (icosahedron, n_sub^2 sub-triangles per face, degree-4 maps onto r(x_hat))
    with 15 nodes each.  Centers and on-surface targets sit at the 15 nodes of every element; the
    sources are those nodes too (upsample = 1), or the 15 f^2 nodes of the rule repeated on the
    f^2 sub-triangles of every element (upsample = f), a finer source quadrature on the same
    elements and expansion radii (the role of the paper's stage-2 quadrature, Section 3)."""
    return surface_from_flat(_flat_subtriangles(n_sub), radius_fn, scale, offset, upsample)


def _element_geometry(flat, radius_fn, scale, offset):
    """(K, 15, 3) geometry nodes: the 15 equispaced points of each flat triangle projected radially
    onto r(x_hat), scaled and shifted."""
    K = flat.shape[0]
    V0, V1, V2 = flat[:, 0], flat[:, 1], flat[:, 2]
    gi = np.array([i for i, _ in _GEO_IJ]) / 4.0
    gj = np.array([j for _, j in _GEO_IJ]) / 4.0
    pts = V0[:, None, :] + gi[None, :, None] * (V1 - V0)[:, None, :] + gj[None, :, None] * (V2 - V0)[:, None, :]
    xhat = pts / np.linalg.norm(pts, axis=-1, keepdims=True)
    rad = radius_fn(xhat.reshape(-1, 3).T).reshape(K, 15)
    return xhat * rad[..., None] * scale + np.asarray(offset)[None, None, :]


def _eta_elements(geo):
    """eta_k: max over the 15 quadrature and 15 geometry nodes of 2 sigma_1(J A^-1) (eq. stretch-factor)."""
    qu, qv, _ = triangle_rule()
    gi = np.array([i for i, _ in _GEO_IJ]) / 4.0
    gj = np.array([j for _, j in _GEO_IJ]) / 4.0
    out = None
    for u, v in ((qu, qv), (gi, gj)):
        _, du_b, dv_b = _lagrange_eval(u, v)
        e = _stretch(np.einsum("qb,kbd->kqd", du_b, geo), np.einsum("qb,kbd->kqd", dv_b, geo)).max(axis=1)
        out = e if out is None else np.maximum(out, e)
    return out


def scaled_curvature(flat: np.ndarray, radius_fn=sphere_radius, scale: float = 1.0,
                     offset=(0.0, 0.0, 0.0)) -> np.ndarray:
    """kappa_k = max over the element's 15 quadrature and 15 geometry nodes x of
    max(|k_1(x)|, |k_2(x)|) eta_k(x) (eq. curvature-criterion, Section 3.2.1): the principal
    curvatures are the eigenvalues of the shape operator I^-1 II of the degree-4 element map,
    eta_k(x) = 2 sigma_1(J A^-1) at x."""
    geo = _element_geometry(flat, radius_fn, scale, offset)
    qu, qv, _ = triangle_rule()
    gi = np.array([i for i, _ in _GEO_IJ]) / 4.0
    gj = np.array([j for _, j in _GEO_IJ]) / 4.0
    u = np.concatenate([qu, gi])
    v = np.concatenate([qv, gj])
    _, du_b, dv_b = _lagrange_eval(u, v)
    uu_b, uv_b, vv_b = _lagrange_eval2(u, v)
    xu = np.einsum("qb,kbd->kqd", du_b, geo)
    xv = np.einsum("qb,kbd->kqd", dv_b, geo)
    xuu = np.einsum("qb,kbd->kqd", uu_b, geo)
    xuv = np.einsum("qb,kbd->kqd", uv_b, geo)
    xvv = np.einsum("qb,kbd->kqd", vv_b, geo)
    n = np.cross(xu, xv)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    E, F, Gm = np.sum(xu * xu, -1), np.sum(xu * xv, -1), np.sum(xv * xv, -1)
    L, M, N = np.sum(xuu * n, -1), np.sum(xuv * n, -1), np.sum(xvv * n, -1)
    # eigenvalues of I^-1 II: k^2 det(I) - k (E N - 2 F M + G L) + det(II) = 0
    detI = E * Gm - F * F
    H2 = (E * N - 2.0 * F * M + Gm * L) / detI        # k1 + k2
    K = (L * N - M * M) / detI                        # k1 k2
    disc = np.sqrt(np.maximum(0.25 * H2 * H2 - K, 0.0))
    kmax = np.maximum(np.abs(0.5 * H2 + disc), np.abs(0.5 * H2 - disc))
    return (kmax * _stretch(xu, xv)).max(axis=1)


def collocation_surface(flat: np.ndarray, radius_fn=sphere_radius, src_degree: int = 10, shrink: float = 0.8,
                        scale: float = 1.0, offset=(0.0, 0.0, 0.0)) -> Surface:
    """Discretization for solving with the evaluation as the operator: the unknowns live at 15 nodes per
    element, the equispaced degree-4 nodes shrunk toward the centroid by `shrink` (interior and
    unisolvent for the polynomials of degree 4, so a density is a degree-4 polynomial per element); the
    centers and on-surface targets sit at those nodes (eq. expansion-centers, r = eta / 2), and the
    sources are the nodes of a node-elimination rule exact to degree src_degree (the oversampled stage-2
    quadrature of Section 3.1), whose density values come from the node values by `interp`."""
    from .rules import eliminated_rule

    K = flat.shape[0]
    geo = _element_geometry(flat, radius_fn, scale, offset)
    gi = np.array([i for i, _ in _GEO_IJ]) / 4.0
    gj = np.array([j for _, j in _GEO_IJ]) / 4.0
    c = 1.0 / 3.0
    nu, nv = c + shrink * (gi - c), c + shrink * (gj - c)
    fu, fv, fw = eliminated_rule(int(src_degree))

    def at(u, v):
        ph, du, dv = _lagrange_eval(u, v)
        return (np.einsum("qb,kbd->kqd", ph, geo), np.einsum("qb,kbd->kqd", du, geo),
                np.einsum("qb,kbd->kqd", dv, geo))

    xn, dun, dvn = at(nu, nv)
    nrm = np.cross(dun, dvn)
    nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    eta = _eta_elements(geo)
    xs, dus, dvs = at(fu, fv)
    crs = np.cross(dus, dvs)
    ars = np.linalg.norm(crs, axis=-1)
    vand = lambda u, v: np.stack([u ** a * v ** b for a, b in _MONO], axis=1)  # noqa: E731
    interp = vand(fu, fv) @ np.linalg.inv(vand(nu, nv))
    node_xyz = np.ascontiguousarray(xn.reshape(-1, 3).T)
    node_n = np.ascontiguousarray(nrm.reshape(-1, 3).T)
    node_elem = np.repeat(np.arange(K, dtype=np.int32), 15)
    r = 0.5 * eta[node_elem]
    N = node_xyz.shape[1]
    ctr = np.concatenate([node_xyz + r * node_n, node_xyz - r * node_n], axis=1)
    return Surface(K, np.ascontiguousarray(xs.reshape(-1, 3).T), np.ascontiguousarray((fw[None, :] * ars).reshape(-1)),
                   np.ascontiguousarray((crs / ars[..., None]).reshape(-1, 3).T),
                   np.repeat(np.arange(K, dtype=np.int32), fu.size), eta, np.ascontiguousarray(ctr),
                   np.concatenate([r, r]), np.concatenate([np.ones(N, np.int8), -np.ones(N, np.int8)]),
                   np.ascontiguousarray(np.concatenate([node_xyz, node_xyz], axis=1)), np.arange(2 * N, dtype=np.int32),
                   radius_fn, np.concatenate([node_elem, node_elem]), eta, interp)


def surface_from_flat(flat: np.ndarray, radius_fn=sphere_radius, scale: float = 1.0, offset=(0.0, 0.0, 0.0),
                      upsample: int = 1, src_flat: np.ndarray = None, src_degree: int = None) -> Surface:
    """Surface on the mesh of flat triangles `flat` (projected radially onto r(x_hat)): the body of
    make_surface for any (e.g. locally bisected) mesh.  With src_flat (a bisection of `flat`: the
    stage-2 mesh of Section 3.3) the sources are the nodes of src_flat's elements (and elem_eta their
    eta), while centers, radii and targets stay those of `flat` (the stage-1 mesh).  With src_degree
    the sources are the nodes of a rule exact to that total degree built by node elimination
    (synth.rules, the stage-2 quadrature of Section 3.1) instead of the 15-node rule (upsample is
    then ignored)."""
    if src_flat is not None:
        s1 = surface_from_flat(flat, radius_fn, scale, offset)
        s2 = surface_from_flat(src_flat, radius_fn, scale, offset, upsample, src_degree=src_degree)
        return Surface(s2.n_elem, s2.src_xyz, s2.src_w, s2.src_n, s2.src_elem, s2.elem_eta, s1.ctr_xyz, s1.ctr_r,
                       s1.ctr_side, s1.tgt_xyz, s1.tgt_ctr, radius_fn, s1.ctr_elem, s1.elem_eta)
    K = flat.shape[0]
    geo = _element_geometry(flat, radius_fn, scale, offset)  # (K, 15, 3)
    gi = np.array([i for i, _ in _GEO_IJ]) / 4.0
    gj = np.array([j for _, j in _GEO_IJ]) / 4.0

    qu, qv, qw = triangle_rule()
    phi, dphu, dphv = _lagrange_eval(qu, qv)  # (15 quad, 15 basis)
    x = np.einsum("qb,kbd->kqd", phi, geo)
    du = np.einsum("qb,kbd->kqd", dphu, geo)
    dv = np.einsum("qb,kbd->kqd", dphv, geo)
    cr = np.cross(du, dv)
    area = np.linalg.norm(cr, axis=-1)
    nrm = cr / area[..., None]
    w = qw[None, :] * area

    # resolution measure: max over quadrature + geometry nodes of the element
    _, gdu, gdv = _lagrange_eval(gi, gj)
    du_g = np.einsum("qb,kbd->kqd", gdu, geo)
    dv_g = np.einsum("qb,kbd->kqd", gdv, geo)
    eta = np.maximum(_stretch(du, dv).max(axis=1), _stretch(du_g, dv_g).max(axis=1))

    node_xyz = np.ascontiguousarray(x.reshape(-1, 3).T)
    node_n = np.ascontiguousarray(nrm.reshape(-1, 3).T)
    node_elem = np.repeat(np.arange(K, dtype=np.int32), 15)
    if upsample > 1 or src_degree is not None:
        if src_degree is not None:
            from .rules import eliminated_rule

            fu, fv, fw = eliminated_rule(int(src_degree))
        else:
            fu, fv, fw = _upsampled_rule(upsample)
        fphi, fdu, fdv = _lagrange_eval(fu, fv)
        xs = np.einsum("qb,kbd->kqd", fphi, geo)
        crs = np.cross(np.einsum("qb,kbd->kqd", fdu, geo), np.einsum("qb,kbd->kqd", fdv, geo))
        ars = np.linalg.norm(crs, axis=-1)
        src_xyz = np.ascontiguousarray(xs.reshape(-1, 3).T)
        src_n = np.ascontiguousarray((crs / ars[..., None]).reshape(-1, 3).T)
        src_w = np.ascontiguousarray((fw[None, :] * ars).reshape(-1))
        src_elem = np.repeat(np.arange(K, dtype=np.int32), fu.size)
    else:
        src_xyz, src_n = node_xyz, node_n
        src_w = np.ascontiguousarray(w.reshape(-1))
        src_elem = node_elem
    r = 0.5 * eta[node_elem]
    N = node_xyz.shape[1]
    ctr = np.concatenate([node_xyz + r * node_n, node_xyz - r * node_n], axis=1)
    ctr_r = np.concatenate([r, r])
    side = np.concatenate([np.ones(N, np.int8), -np.ones(N, np.int8)])
    tgt = np.concatenate([node_xyz, node_xyz], axis=1)
    tctr = np.arange(2 * N, dtype=np.int32)
    return Surface(K, src_xyz, src_w, src_n, src_elem, eta, np.ascontiguousarray(ctr), ctr_r, side,
                   np.ascontiguousarray(tgt), tctr, radius_fn, np.concatenate([node_elem, node_elem]), eta)


# --------------------------------------------------------------------------
# densities and off-surface targets
# --------------------------------------------------------------------------


def greens_density(surf: Surface, x0=(3.0, 1.0, 2.0)):
    """u = 1/|x - x0| and its outward normal derivative at the sources.

    Green's formula (Section 6.1): S(d_n u) - D(u) = u/2 on the surface for u
    harmonic inside.  Returns (u, dudn) at the sources.
    """
    d = surf.src_xyz - np.asarray(x0)[:, None]
    rr = np.sqrt(np.sum(d * d, axis=0))
    u = 1.0 / rr
    dudn = -np.sum(surf.src_n * d, axis=0) / rr ** 3
    return u, dudn


def random_harmonic_density(surf: Surface, nmax: int = 10, seed: int = 4):
    """sum over n <= nmax, real basis index m, of c_nm Y~_n^m(x_hat), c_nm ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    xhat = surf.src_xyz / np.linalg.norm(surf.src_xyz, axis=0)
    out = np.zeros(surf.n_src)
    for n in range(nmax + 1):
        for m in range(-n, n + 1):
            out += rng.standard_normal() * real_ylm(n, m, xhat)
    return out


def danger_radius(surf: Surface) -> np.ndarray:
    """Radius of the danger zone around each source node, eta_k / 2 of its element (Section 3.4)."""
    return 0.5 * surf.elem_eta[surf.src_elem]


def volume_points(n: int = 10000, seed: int = 2, box: float = 2.0) -> np.ndarray:
    """Seeded points uniform in [-box, box]^3, (3, n)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.uniform(-box, box, size=(n, 3)).T)


def near_surface_points(surf: Surface, n: int, seed: int = 3, spread: float = 2.0) -> np.ndarray:
    """Seeded points near the surface: a random source node moved along its normal by a uniform
    multiple in [-spread, spread] of its danger radius, plus a tangential jitter of the same size
    (so that many points are endangered and both sides are represented), (3, n)."""
    rng = np.random.default_rng(seed)
    j = rng.integers(0, surf.n_src, n)
    rd = danger_radius(surf)[j]
    x = surf.src_xyz[:, j] + surf.src_n[:, j] * (rng.uniform(-spread, spread, n) * rd)
    x = x + rng.normal(size=(3, n)) * (0.5 * rd)
    return np.ascontiguousarray(x)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

STAR_Y63 = [(0.3, 6, 3)]
STAR_Y84_Y52 = [(0.25, 8, 4), (0.15, 5, 2)]


def batched_specs(count: int = 64, seed: int = 5):
    """Specs of the many-surface workload: star surfaces r = 1 + a Re Y_k^{floor(k/2)} with
    k ~ U{2..10}, a ~ U[0.1, 0.4], and source counts N ~ lognormal(10.36, 0.941) clipped to
    [5k, 200k], realised as 300 n^2 sources (n = round(sqrt(N / 300)) in [4, 26]).  Returns a list
    of (n_sub, terms, density_seed) with density seeds 500 + i for random_harmonic_density."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        k = int(rng.integers(2, 11))
        a = float(rng.uniform(0.1, 0.4))
        n_target = float(np.clip(rng.lognormal(10.36, 0.941), 5000.0, 200000.0))
        n = int(np.clip(round(math.sqrt(n_target / 300.0)), 4, 26))
        out.append((n, [(a, k, k // 2)], 500 + i))
    return out


def config_surface(name: str) -> Surface:
    """Surfaces of the named workloads: sphere320, star8k, star40k, urchin79k."""
    if name == "sphere320":
        return make_surface(4, sphere_radius)
    if name == "star8k":
        return make_surface(20, star_radius(STAR_Y63))
    if name == "star40k":
        return make_surface(45, star_radius(STAR_Y63))
    if name == "star79k":
        return make_surface(63, star_radius(STAR_Y84_Y52))
    raise KeyError(name)
