"""Pins of the oracle's Clenshaw-Curtis pair and region rule (Sec. 3).

The rule is pinned against the N = 4 weights printed in the CC literature,
the moment equations of interpolatory quadrature solved independently, the
nesting property that the paper relies on (the N points are a subset of the
2N points), and polynomial exactness of the 2-D tensor rule on whole and
partial domains.
"""
import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
LAT = (1.0, -0.25, -1.0)


def test_cc_n4_matches_golden():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "cc_weights_n4.txt"))
            if l.strip() and not l.startswith("#")]
    want = np.array([int(r[1]) / int(r[2]) for r in rows])
    x, w = oracle.cc_rule(4)
    assert np.allclose(w, want, rtol=0, atol=1e-15)
    assert np.allclose(x, [1, math.sqrt(0.5), 0, -math.sqrt(0.5), -1], atol=1e-15)


@pytest.mark.parametrize("N", [2, 4, 6, 8, 12, 16, 24, 32])
def test_cc_weights_solve_moment_equations(N):
    x, w = oracle.cc_rule(N)
    # interpolatory on N+1 nodes: exact for every polynomial of degree <= N.
    # Solve the moment equations independently, in the well-conditioned
    # Chebyshev basis: int_{-1}^{1} T_k = 2/(1-k^2) for even k, 0 for odd k.
    V = np.vstack([np.polynomial.chebyshev.chebval(x, np.eye(N + 1)[k]) for k in range(N + 1)])
    mu = np.array([2.0 / (1 - k * k) if k % 2 == 0 else 0.0 for k in range(N + 1)])
    w_ref = np.linalg.solve(V, mu)
    assert np.allclose(w, w_ref, rtol=0, atol=1e-12)
    assert abs(w.sum() - 2.0) < 1e-14
    assert np.allclose(w, w[::-1], atol=1e-15)
    # N even: the symmetric rule is also exact for degree N+1, not N+2
    assert abs(np.dot(w, x ** (N + 1))) < 1e-14
    if N <= 24:
        assert abs(np.dot(w, x ** (N + 2)) - 2.0 / (N + 3)) > 1e-12


@pytest.mark.parametrize("N", [2, 4, 6, 8])
def test_coarse_nodes_are_even_fine_nodes(N):
    xc, _ = oracle.cc_rule(N)
    xf, _ = oracle.cc_rule(2 * N)
    assert np.allclose(xc, xf[::2], atol=1e-15)


def _exact_monomial(a, b, L, ix, iy):
    """(1/(2pi)^2) * int over the region of (x/pi)^a (y/pi)^b, in closed form."""
    h = 2 * math.pi / 2 ** L
    x0, x1 = -math.pi + ix * h, -math.pi + (ix + 1) * h
    y0, y1 = -math.pi + iy * h, -math.pi + (iy + 1) * h
    ix_ = (x1 ** (a + 1) - x0 ** (a + 1)) / ((a + 1) * math.pi ** a)
    iy_ = (y1 ** (b + 1) - y0 ** (b + 1)) / ((b + 1) * math.pi ** b)
    return ix_ * iy_ / (4 * math.pi ** 2)


@pytest.mark.parametrize("L,ix,iy", [(0, 0, 0), (1, 1, 0), (2, 3, 1), (3, 5, 2)])
def test_region_rule_polynomial_exactness(L, ix, iy):
    for a in range(0, 12):
        for b in range(0, 12):
            qN, q2N = oracle.region_eval(oracle.MONOMIAL, (0.0, 0.0), a, b, 1.0, LAT, L, ix, iy)
            ex = _exact_monomial(a, b, L, ix, iy)
            scale = max(1.0, abs(ex)) * 1e-14
            if a <= 9 and b <= 9:
                assert abs(q2N - ex) < scale, (a, b, q2N, ex)
            if a <= 5 and b <= 5:
                assert abs(qN - ex) < scale, (a, b, qN, ex)
                assert abs(qN - q2N) < scale
    # degree 10 in x breaks the fine rule on the whole domain: the degree is not higher
    qN, q2N = oracle.region_eval(oracle.MONOMIAL, (0.0, 0.0), 10, 0, 1.0, LAT, 0, 0, 0)
    assert abs(q2N - _exact_monomial(10, 0, 0, 0, 0)) > 1e-6
    # degree 6 breaks the coarse rule, so err > 0 there
    qN, q2N = oracle.region_eval(oracle.MONOMIAL, (0.0, 0.0), 6, 0, 1.0, LAT, 0, 0, 0)
    assert abs(qN - q2N) > 1e-4


def test_adaptive_monomials_reach_closed_form():
    lm = np.array([(a, b) for a in range(0, 13) for b in range(0, 13)], dtype=np.int32)
    q = np.zeros((1, 2))
    v, e, r, s = oracle.integrate_batch(oracle.MONOMIAL, q, lm, 1.0, LAT, 1e-10, 1e-14, 20000,
                                        init_level=0)
    for i, (a, b) in enumerate(lm):
        ex = 1.0 / ((a + 1) * (b + 1)) if (a % 2 == 0 and b % 2 == 0) else 0.0
        assert s[i] == oracle.CONVERGED
        assert abs(v[i] - ex) <= max(e[i], 1e-15) + 1e-15, (a, b, v[i], ex, e[i])
        if a <= 5 and b <= 5:
            assert r[i] == 1  # coarse rule exact: one region suffices


def test_invalid_rule_rejected():
    with pytest.raises(ValueError):
        oracle.cc_rule(3)
    with pytest.raises(ValueError):
        oracle.region_eval(oracle.PH, (0.0, 0.0), 0, 0, 0.5, LAT, 0, 0, 0, rule_n=5)
