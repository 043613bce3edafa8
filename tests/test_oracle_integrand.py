"""Pins of the oracle's integrand pieces (Sec. 2, Eq. chi_ph / chi_pp in
Matsubara-summed temperature form).

* form factors: orthonormality (Gram = I at q = 0) and the closed-form shift
  matrix at q != 0, through the OVERLAP kind and the adaptive driver;
* the ph / pp kernels: a 50-digit evaluation of the direct definition with
  mpmath at random points, the analytic limits at a vanishing denominator,
  continuity across the oracle's internal branch, and the high-T limit;
* the dispersion against its formula at random points.
"""
import math

import numpy as np
import pytest

import oracle
from tests import np_ref

mp = pytest.importorskip("mpmath")
LAT = (1.0, -0.25, -1.0)


def test_shift_matrix_is_pointwise_identity():
    # the hand-derived S(q) itself, checked at random k (guards the pin)
    rng = np.random.default_rng(3)
    for _ in range(5):
        q = rng.uniform(-math.pi, math.pi, 2)
        S = np_ref.shift_matrix(q)
        k = rng.uniform(-math.pi, math.pi, (50, 2))
        F = np.stack([np_ref.ff(n, k[:, 0], k[:, 1]) for n in range(9)], 1)
        Fs = np.stack([np_ref.ff(n, k[:, 0] + q[0], k[:, 1] + q[1]) for n in range(9)], 1)
        assert np.allclose(Fs, F @ S.T, atol=1e-13)


def test_form_factors_match_numpy():
    rng = np.random.default_rng(5)
    for _ in range(40):
        kx, ky = rng.uniform(-4, 4, 2)
        for n in range(9):
            assert abs(oracle.form_factor(n, kx, ky) - float(np_ref.ff(n, kx, ky))) < 1e-15
    assert math.isnan(oracle.form_factor(9, 0.1, 0.2))


@pytest.mark.parametrize("q", [(0.0, 0.0), (0.7, -1.9), (math.pi, math.pi), (-2.5, 0.4)])
def test_overlap_gram_equals_shift_matrix(q):
    lm = np.array([(l, m) for l in range(9) for m in range(9)], dtype=np.int32)
    v, e, r, s = oracle.integrate_batch(oracle.OVERLAP, np.array([q]), lm, 1.0, LAT,
                                        1e-12, 1e-12, 20000, init_level=0)
    assert np.all(s == oracle.CONVERGED)
    G = v.reshape(9, 9)
    want = np_ref.shift_matrix(q).T  # <f_l, f_m(. + q)> = S[m, l]
    assert np.all(np.abs(G - want) <= e.reshape(9, 9) + 1e-13)
    assert np.allclose(G, want, atol=2e-12)
    if q == (0.0, 0.0):
        assert np.allclose(G, np.eye(9), atol=2e-13)


def _mp_kernel(kind, e1, e2, T):
    mp.mp.dps = 50
    e1, e2, T = mp.mpf(e1), mp.mpf(e2), mp.mpf(T)
    nf = lambda e: 1 / (mp.exp(e / T) + 1)
    if kind == 0:
        if e1 == e2:
            return -mp.diff(nf, e1)
        return (nf(e2) - nf(e1)) / (e1 - e2)
    if e1 == -e2:
        return -mp.diff(nf, e1)
    return (1 - nf(e1) - nf(e2)) / (e1 + e2)


def _cases(seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(120):
        T = float(np.exp(rng.uniform(math.log(0.005), math.log(2.0))))
        e1 = float(rng.uniform(-6, 6))
        mode = rng.integers(0, 4)
        if mode == 0:
            e2 = float(rng.uniform(-6, 6))
        elif mode == 1:
            e2 = e1 + float(rng.choice([-1, 1]) * 10.0 ** rng.uniform(-14, -1)) * T
        elif mode == 2:
            e2 = e1
        else:
            e2 = e1 + float(rng.uniform(-2.5, 2.5)) * T
        out.append((e1, e2, T))
    return out


@pytest.mark.parametrize("kind", [0, 1])
def test_kernel_against_50_digit_definition(kind):
    f = oracle.kernel_ph if kind == 0 else oracle.kernel_pp
    for e1, e2, T in _cases(11 + kind):
        if kind == 1:
            e2 = -e2  # pp is degenerate at e1 + e2 = 0
        got = f(e1, e2, T)
        want = float(_mp_kernel(kind, e1, e2, T))
        peak = 1.0 / (4.0 * T)
        # relative where the value matters, absolute against the kernel's scale elsewhere
        assert abs(got - want) <= 1e-13 * abs(want) + 1e-15 * peak, (kind, e1, e2, T, got, want)


@pytest.mark.parametrize("kind", [0, 1])
def test_kernel_limits_and_branch_continuity(kind):
    f = oracle.kernel_ph if kind == 0 else oracle.kernel_pp
    sgn = 1.0 if kind == 0 else -1.0
    for T in (0.005, 0.05, 0.5):
        for e in (-0.3, 0.0, 0.01, 2.0):
            lim = 1.0 / (4.0 * T * math.cosh(e / (2 * T)) ** 2)
            assert abs(f(e, sgn * e, T) - lim) <= 1e-15 * lim + 1e-300
            # continuity into the limit from both sides
            for d in (1e-12, -1e-9):
                v = f(e, sgn * (e + d), T)
                assert abs(v - lim) <= 1e-6 * lim
            # across the oracle's branch at |x1 -+ x2| = 1
            for side in (1.0, -1.0):
                e2 = e + side * 2.0 * T
                a = f(e, sgn * (e2 * (1 - 1e-13)), T)
                b = f(e, sgn * (e2 * (1 + 1e-13)), T)
                assert abs(a - b) <= 1e-10 * abs(a) + 1e-300


@pytest.mark.parametrize("kind", [0, 1])
def test_kernel_high_temperature_limit(kind):
    f = oracle.kernel_ph if kind == 0 else oracle.kernel_pp
    T = 1e5
    for e1, e2 in [(0.3, -1.2), (2.0, 2.5), (-4.0, 1.0)]:
        assert abs(4.0 * T * f(e1, e2, T) - 1.0) < 1e-9


def test_dispersion_formula():
    rng = np.random.default_rng(1)
    for _ in range(30):
        kx, ky = rng.uniform(-4, 4, 2)
        t, tp, mu = rng.uniform(-2, 2, 3)
        want = -2 * t * (math.cos(kx) + math.cos(ky)) - 4 * tp * math.cos(kx) * math.cos(ky) - mu
        assert abs(oracle.dispersion(kx, ky, t, tp, mu) - want) < 1e-14


def test_integrand_composition_matches_numpy_at_points():
    rng = np.random.default_rng(9)
    for kind in (0, 1, 2, 3):
        for _ in range(30):
            q = tuple(rng.uniform(-math.pi, math.pi, 2))
            l, m = (int(x) for x in rng.integers(0, 9, 2))
            T = float(rng.uniform(0.05, 1.0))
            kx, ky = rng.uniform(-math.pi, math.pi, 2)
            got = oracle.integrand_point(kind, q, l, m, T, LAT, kx, ky)
            want = float(np_ref.integrand(kind, q, l, m, T, LAT, np.float64(kx), np.float64(ky)))
            assert abs(got - want) <= 1e-12 * abs(want) + 1e-14, (kind, q, l, m, T, got, want)
