"""Pins of the node-elimination quadrature rules (synth.rules; the construction the paper's stage-2
quadrature uses, Section 3.1), no GPU: exactness on every monomial of the triangle up to the rule's
degree (integrals a! b! / (a + b + 2)!), inexactness one degree up, nodes inside and weights
positive, fewer nodes than the conical rule they start from, and as the sources of a surface a
smooth integral over the discretized sphere more accurate than with the 15-node rule on the same mesh."""
import math

import numpy as np
import pytest

from synth import flat_mesh, surface_from_flat
from synth.rules import eliminated_rule, exactness_error


@pytest.mark.parametrize("d", [5, 8, 10])
def test_eliminated_rules(d):
    u, v, w = eliminated_rule(d)
    assert exactness_error(u, v, w, d) < 1e-15
    worst = max(abs(float(np.sum(w * u ** a * v ** (d + 1 - a))) - math.factorial(a) * math.factorial(d + 1 - a) /
                    math.factorial(d + 3)) for a in range(d + 2))
    assert worst > 1e-9
    assert np.all(u > 0) and np.all(v > 0) and np.all(u + v < 1) and np.all(w > 0)
    assert len(u) < ((d + 2) // 2) ** 2


def test_rule_as_stage2_sources():
    f = flat_mesh(3)
    s15 = surface_from_flat(f)
    s10 = surface_from_flat(f, src_degree=10)
    assert s10.n_src == 25 * s15.n_elem and s10.n_ctr == s15.n_ctr
    # int of z^2 over the discretized surface (the degree-4 element maps), by a much finer rule on it
    ref = surface_from_flat(f, upsample=8)
    exact = np.sum(ref.src_w * ref.src_xyz[2] ** 2)
    e15 = abs(np.sum(s15.src_w * s15.src_xyz[2] ** 2) - exact)
    e10 = abs(np.sum(s10.src_w * s10.src_xyz[2] ** 2) - exact)
    assert e10 < 0.1 * e15
