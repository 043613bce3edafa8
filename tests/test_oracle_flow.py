"""Pins of the oracle's Omega-regulated flow kernels and integrals (Sec. 2:
G(k) = theta(k0) / (i k0 - e(k)), theta = k0^2 / (k0^2 + Omega^2); the inner
frequency integrals of Eqs. chi_ph / chi_pp, differentiated in Omega).

The closed forms are held to a numerical quadrature of their definition,
  d/dOmega int dk0/2pi theta(k0)^2 / ((i k0 - e1)(i k0 - e2))            (ph)
  d/dOmega int dk0/2pi theta(k0) theta(-k0) / ((i k0 - e1)(-i k0 - e2))  (pp)
(the Omega derivative taken under the integral), at random, near-degenerate,
opposite-sign and zero energies; the 2-D integrals to a converged dense
trapezoid; plus the symmetries of the symmetric routing."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1610_09991_gb300 import workloads as W

LAT = W.LATTICE


def _quad(e1, e2, om, pp):
    def f(k0):
        if k0 == 0.0:
            return 0.0   # d theta^2 / dOmega vanishes like k0^4 there
        dtheta2 = -4.0 * om * k0 ** 4 / (k0 * k0 + om * om) ** 3
        if pp:
            g = 1.0 / ((1j * k0 - e1) * (-1j * k0 - e2))
        else:
            g = 1.0 / ((1j * k0 - e1) * (1j * k0 - e2))
        return dtheta2 * g.real
    pts = sorted({om} | {abs(x) for x in (e1, e2) if abs(x) > 1e-9})
    a = 0.0
    total = 0.0
    for b in pts + [math.inf]:
        if b > a:
            v, _ = integrate.quad(f, a, b, limit=400, epsabs=0.0, epsrel=1e-13)
            total += v
            a = b
    return 2.0 * total / (2.0 * math.pi)   # even integrand, measure dk0 / 2pi


CASES = [(0.7, -0.3, 0.5), (0.4, 0.4000001, 0.2), (-1.3, -1.29, 0.05), (0.0, 0.8, 0.3),
         (0.0, 0.0, 0.1), (2.5, -3.1, 1.0), (-0.02, 0.03, 0.01), (5.0, 5.0, 0.02),
         (1e-3, -1e-3, 0.5), (-4.0, -0.5, 2.0)]


@pytest.mark.parametrize("e1,e2,om", CASES)
def test_flow_kernels_match_frequency_quadrature(e1, e2, om):
    for pp in (False, True):
        want = _quad(e1, e2, om, pp)
        got = oracle.kernel_flow_pp(e1, e2, om) if pp else oracle.kernel_flow_ph(e1, e2, om)
        assert abs(got - want) <= 1e-9 * max(abs(want), 1e-3 / om ** 2), (e1, e2, om, pp, got, want)


def test_flow_kernel_random_points():
    rng = np.random.default_rng(11)
    for _ in range(60):
        e1, e2 = rng.normal(scale=1.5, size=2)
        om = 10 ** rng.uniform(-2, 0.5)
        for pp in (False, True):
            want = _quad(e1, e2, om, pp)
            got = oracle.kernel_flow_pp(e1, e2, om) if pp else oracle.kernel_flow_ph(e1, e2, om)
            assert abs(got - want) <= 1e-9 * max(abs(want), 1e-3 / om ** 2)


def test_flow_kernel_symmetry_and_limits():
    # ph is symmetric in (e1, e2); the degenerate limit is the derivative of Hdot
    for e, om in [(0.3, 0.2), (-1.1, 0.05), (0.0, 0.7)]:
        a = oracle.kernel_flow_ph(e, e + 1e-7, om)
        b = oracle.kernel_flow_ph(e, e, om)
        assert abs(a - b) <= 1e-5 * abs(b)
        assert oracle.kernel_flow_ph(e, 0.4, om) == oracle.kernel_flow_ph(0.4, e, om)
    # at e1 = e2 = 0 the ph kernel is 1 / (4 Omega^2)
    assert abs(oracle.kernel_flow_ph(0.0, 0.0, 0.3) - 1.0 / (4 * 0.09)) < 1e-14


@pytest.mark.parametrize("kind", [oracle.FLOW_PH, oracle.FLOW_PP])
def test_flow_integrals_against_trapezoid(kind):
    q = np.array([(0.9, -0.4), (math.pi, 0.0)])
    lm = np.array([(0, 0), (1, 1), (2, 5), (3, 3), (6, 8)], dtype=np.int32)
    om = 0.2
    # (6, 8) vanishes by inversion symmetry: the absolute floor decides it
    v, e, r, s = oracle.integrate_batch(kind, q, lm, om, LAT, 1e-9, 1e-11, 100000)
    assert np.all(s == oracle.CONVERGED)
    for iq in range(2):
        for ip, (l, m) in enumerate(lm):
            i = iq * len(lm) + ip
            # the kernel's fourth derivative jumps on the Fermi surface, so the
            # periodic trapezoid converges like h^4 there (measured ratio ~15.6
            # per halving): one Richardson step on M = 2048, 4096
            t1 = oracle.trapezoid(kind, q[iq], l, m, om, LAT, 2048)
            t2 = oracle.trapezoid(kind, q[iq], l, m, om, LAT, 4096)
            assert abs(t1 - t2) < 5e-11
            tr = t2 + (t2 - t1) / 15.0
            assert abs(v[i] - tr) <= e[i] + 2e-12
    assert np.all(np.abs(v.reshape(2, -1)[:, 4]) < 1e-11)


def test_flow_brute_force_extrapolates():
    # the decider the bench uses for the flow kinds: Richardson-extrapolated
    # trapezoid against a tight adaptive value; the plain doubling test of
    # brute_force would never reach 1e-13 on these integrands
    q = np.array([(0.9, -0.4)])
    v, e, r, s = oracle.integrate_batch(oracle.FLOW_PH, q, np.array([(2, 5)]), 0.2, LAT,
                                        1e-10, 1e-13, 1000000)
    assert s[0] == oracle.CONVERGED
    bf, M = oracle.brute_force(oracle.FLOW_PH, q[0], 2, 5, 0.2, LAT)
    assert M <= 16384 and abs(bf - v[0]) <= e[0] + 2e-11


def test_flow_routing_symmetries():
    # f_m(k) f_n(k): I_mn = I_nm; l -> -l swaps the two energies: I(-l) = I(l)
    lm = W.all_pairs(9)
    q = np.array([(1.1, 0.45), (-1.1, -0.45)])
    for kind in (oracle.FLOW_PH, oracle.FLOW_PP):
        v, e, r, s = oracle.integrate_batch(kind, q, lm, 0.3, LAT, 1e-10, 1e-13, 100000)
        I, E = v.reshape(2, 9, 9), e.reshape(2, 9, 9)
        assert np.all(np.abs(I[0] - I[0].T) <= E[0] + E[0].T + 1e-13)
        if kind == oracle.FLOW_PH:
            assert np.all(np.abs(I[0] - I[1]) <= E[0] + E[1] + 1e-13)


def _bubble_quad(e1, e2, om):
    """int dk0/2pi theta(k0)^2 / ((i k0 - e1)(i k0 - e2)): the ph bubble's
    frequency integral itself (no derivative)."""
    def f(k0):
        th = k0 * k0 / (k0 * k0 + om * om)
        return (th * th / ((1j * k0 - e1) * (1j * k0 - e2))).real
    pts = sorted({om} | {abs(x) for x in (e1, e2) if abs(x) > 1e-9})
    a, total = 0.0, 0.0
    for b in pts + [math.inf]:
        if b > a:
            v, _ = integrate.quad(f, a, b, limit=400, epsabs=0.0, epsrel=1e-13)
            total += v
            a = b
    return 2.0 * total / (2.0 * math.pi)


@pytest.mark.parametrize("e1,e2,om", [(0.7, -0.3, 0.5), (-1.3, -1.29, 0.2), (0.0, 0.8, 0.3),
                                      (2.5, -3.1, 1.0)])
def test_flow_kernel_is_the_omega_derivative_of_the_bubble(e1, e2, om):
    # the TU flow equations (Eqs. matmul-P/C/D) take the derivative of the
    # bubble of Eqs. chi_pp / chi_ph; the text after the T-equations says the
    # frequency integrals are the Omega derivative of a product of two
    # propagators.  A central difference of the undifferentiated bubble pins
    # that reading (the regulators of both propagators vary), independently
    # of differentiating under the integral
    h = 1e-4 * om
    fd = (_bubble_quad(e1, e2, om + h) - _bubble_quad(e1, e2, om - h)) / (2 * h)
    got = oracle.kernel_flow_ph(e1, e2, om)
    assert abs(got - fd) <= 1e-6 * max(abs(fd), 1e-3 / om ** 2)
    # the single-scale reading (only one propagator's regulator varies) is
    # half of it for the ph bubble's symmetric frequency integrand
    def half(k0):
        if k0 == 0.0:
            return 0.0
        th = k0 * k0 / (k0 * k0 + om * om)
        dth = -2.0 * om * k0 * k0 / (k0 * k0 + om * om) ** 2
        return (dth * th / ((1j * k0 - e1) * (1j * k0 - e2))).real
    v, _ = integrate.quad(half, 0, math.inf, limit=400, epsabs=0.0, epsrel=1e-12)
    assert abs(2 * v / (2 * math.pi) - 0.5 * got) <= 1e-6 * max(abs(got), 1e-3 / om ** 2)
