"""Pins of the oracle's full adaptive integrals (Algorithm 1 over the
Sec. 2 integrands) against brute force, symmetry and special cases.

* dense periodic trapezoid (M doubled to convergence) and tensor
  Gauss-Legendre brute force at high T on every integral of the 400-integral
  first-shell batch, and trapezoid on a seeded sample at T = 0.05;
* the C4v point group and q -> -q relations of the bubbles;
* the nesting identity at t' = 0, mu = 0 and the compressibility identity
  ph_00(q = 0) = d rho / d mu;
* the high-T limit I -> (1/4T) Gram(q).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1610_09991_gb300 import workloads as W
from tests import np_ref

LAT = W.LATTICE


def _ok(v, ref, rel, ab, e=0.0):
    return abs(v - ref) <= max(rel * abs(ref), ab) + e


def test_first_shell_batch_against_trapezoid_and_gauss_legendre():
    w = W.config_first_shell()
    b = w.batches[0]
    v, e, r, s = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol,
                                        b.max_regions)
    assert np.all(s == oracle.CONVERGED)
    worst = 0.0
    for iq in range(b.q.shape[0]):
        for ip, (l, m) in enumerate(b.lm):
            i = iq * b.lm.shape[0] + ip
            t1 = np_ref.trapezoid(b.kind, b.q[iq], l, m, b.T, LAT, 128)
            t2 = np_ref.trapezoid(b.kind, b.q[iq], l, m, b.T, LAT, 256)
            assert abs(t1 - t2) < 1e-14  # converged brute force
            # the adaptive result lies within its own error estimate of the truth
            assert abs(v[i] - t2) <= e[i] + 1e-14, (iq, l, m, v[i], t2, e[i])
            worst = max(worst, abs(v[i] - t2) / max(abs(t2), 1e-4))
    assert worst < 1e-6
    # tensor Gauss-Legendre (not spectrally exact for periodic functions, so
    # converged by size) on a few of them
    for iq, ip in [(0, 0), (5, 6), (10, 12), (15, 24), (7, 18)]:
        l, m = b.lm[ip]
        g = np_ref.gauss_legendre(b.kind, b.q[iq], l, m, b.T, LAT, 160)
        g2 = np_ref.gauss_legendre(b.kind, b.q[iq], l, m, b.T, LAT, 240)
        assert abs(g - g2) < 1e-13
        assert abs(v[iq * 25 + ip] - g2) <= e[iq * 25 + ip] + 1e-13


@pytest.mark.parametrize("kind", [0, 1])
def test_high_T_pp_and_ph_against_trapezoid(kind):
    q = np.array([(0.4, -2.2), (math.pi, 0.0), (-1.3, 2.9)])
    lm = W.all_pairs(9)[::4]
    v, e, r, s = oracle.integrate_batch(kind, q, lm, 1.0, LAT, 1e-8, 1e-12, 100000)
    assert np.all(s == oracle.CONVERGED)
    for iq in range(3):
        for ip, (l, m) in enumerate(lm):
            i = iq * lm.shape[0] + ip
            tr = np_ref.trapezoid(kind, q[iq], l, m, 1.0, LAT, 128)
            assert abs(v[i] - tr) <= e[i] + 1e-14


@pytest.mark.slow
def test_low_T_sample_against_trapezoid():
    # T = 0.05: seeded sample of the 93,312-integral flow-step batch
    w = W.config_flow_step()
    flat = W.flatten(w)
    idx = W.sample_indices(w.n, 6, seed=1234)
    v, e, r, s = oracle.integrate_list(flat["kind"][idx], flat["q"][idx], flat["lm"][idx],
                                       flat["T"][idx], LAT, 1e-6, 1e-10, 100000)
    for j, i in enumerate(idx):
        kind, q, (l, m), T = flat["kind"][i], flat["q"][i], flat["lm"][i], flat["T"][i]
        t1 = np_ref.trapezoid(kind, q, l, m, T, LAT, 1024)
        t2 = np_ref.trapezoid(kind, q, l, m, T, LAT, 2048)
        assert abs(t1 - t2) < 1e-12
        assert abs(v[j] - t2) <= e[j] + 1e-12, (kind, q, l, m, v[j], t2, e[j])


def _grid_T05(kind, qs):
    lm = W.all_pairs(9)
    v, e, r, s = oracle.integrate_batch(kind, np.array(qs), lm, 0.5, LAT, 1e-9, 1e-13, 100000)
    assert np.all(s == oracle.CONVERGED)
    return v.reshape(len(qs), 9, 9), e.reshape(len(qs), 9, 9)


@pytest.mark.parametrize("kind", [0, 1])
def test_c4v_covariance(kind):
    q0 = np.array([0.9, -0.35])
    ops = np_ref.c4v_ops()
    qs = [tuple(g @ q0) for g in ops]
    I, E = _grid_T05(kind, qs)
    for j, g in enumerate(ops):
        D = np_ref.ff_rep(g)
        assert np.allclose(D @ D.T, np.eye(9), atol=1e-12)  # signed permutation
        want = D @ I[0] @ D.T
        tol = 2 * np.maximum(1e-9 * np.abs(want), 1e-13) + E[j] + E[0]
        assert np.all(np.abs(I[j] - want) <= tol), (kind, g)


def test_q_inversion_relations():
    q = (1.1, 0.45)
    mq = (-1.1, -0.45)
    Iph, Eph = _grid_T05(0, [q, mq])
    Ipp, Epp = _grid_T05(1, [q, mq])
    P = np.outer(np_ref.PARITY, np_ref.PARITY)
    tol_ph = Eph[0] + Eph[1] + 1e-13
    tol_pp = Epp[0] + Epp[1] + 1e-13
    # ph: I_lm(-q) = I_ml(q) and I_lm(-q) = p_l p_m I_lm(q)
    assert np.all(np.abs(Iph[1] - Iph[0].T) <= tol_ph + tol_ph.T)
    assert np.all(np.abs(Iph[1] - P * Iph[0]) <= tol_ph)
    # pp: I_lm = I_ml, and the same parity relation
    assert np.all(np.abs(Ipp[0] - Ipp[0].T) <= Epp[0] + Epp[0].T + 1e-13)
    assert np.all(np.abs(Ipp[1] - P * Ipp[0]) <= tol_pp)


def test_nesting_identity_at_half_filling():
    # t' = 0, mu = 0: e(k + Q) = -e(k), so ph_lm(Q) = s_m p_m pp_lm(0)
    lat = (1.0, 0.0, 0.0)
    lm = W.all_pairs(9)
    Q = np.array([(math.pi, math.pi)])
    Z = np.array([(0.0, 0.0)])
    vph, eph, _, sph = oracle.integrate_batch(0, Q, lm, 0.3, lat, 1e-9, 1e-13, 100000)
    vpp, epp, _, spp = oracle.integrate_batch(1, Z, lm, 0.3, lat, 1e-9, 1e-13, 100000)
    assert np.all(sph == 0) and np.all(spp == 0)
    sign = np.outer(np.ones(9), np_ref.SHIFT_Q * np_ref.PARITY).reshape(-1)
    assert np.all(np.abs(vph - sign * vpp) <= eph + epp + 1e-13)
    # and it is not trivially satisfied
    assert np.abs(vph).max() > 0.05


def test_compressibility_identity():
    # ph_00(q = 0) = -(1/(2pi)^2) int nF'(e) = d rho / d mu
    T = 0.4
    v, e, _, s = oracle.integrate_batch(0, np.zeros((1, 2)), np.array([(0, 0)]), T, LAT,
                                        1e-10, 1e-14, 100000)
    t, tp, mu = LAT
    h = 1e-4
    M = 256

    def rho(mu_):
        g = -math.pi + 2 * math.pi * np.arange(M) / M
        KX, KY = np.meshgrid(g, g, indexing="ij")
        return float(np.mean(np_ref.nF(np_ref.disp(KX, KY, (t, tp, mu_)), T)))

    drho = (rho(mu + h) - rho(mu - h)) / (2 * h)
    assert abs(v[0] - drho) < 1e-8 + e[0]


def test_high_T_limit_is_gram_over_4T():
    T = 1e4
    q = (0.8, -2.1)
    lm = W.all_pairs(9)
    v, e, _, s = oracle.integrate_batch(0, np.array([q]), lm, T, LAT, 1e-12, 1e-16, 100000,
                                        init_level=0)
    G = np_ref.shift_matrix(q).T
    assert np.allclose(4 * T * v.reshape(9, 9), G, atol=1e-6)


def test_brute_force_trapezoid_matches_numpy():
    # the oracle's dense trapezoid against the independent numpy restatement
    for kind, q, l, m, T in [(0, (0.3, 1.1), 2, 5, 0.5), (1, (-2.0, 0.7), 8, 3, 0.2)]:
        a = oracle.trapezoid(kind, q, l, m, T, LAT, 96)
        b = np_ref.trapezoid(kind, q, l, m, T, LAT, 96)
        assert abs(a - b) < 1e-15
    v, M = oracle.brute_force(0, (0.3, 1.1), 2, 5, 0.5, LAT, M0=64)
    assert np.isfinite(v) and M <= 256


def test_heuristic_error_estimate_can_miss():
    # Sec. 3's err = |Q_N - Q_2N| is an estimate: on this ph integral at T = 0.05
    # the greedy order stops with a true error 4x its error sum.  Parity
    # disagreements are therefore decided by the converged brute force.
    q = (math.pi / 6, 5 * math.pi / 6)
    v, e, r, s = oracle.integrate_batch(0, np.array([q]), np.array([(1, 7)]), 0.05, LAT,
                                        1e-6, 1e-10, 100000)
    truth, M = oracle.brute_force(0, q, 1, 7, 0.05, LAT)
    assert s[0] == oracle.CONVERGED and np.isfinite(truth)
    assert abs(v[0] - truth) > 2 * e[0]
    assert abs(v[0] - truth) < 1e-7


def _ph00_q0(T, lat):
    v, e, _, s = oracle.integrate_batch(0, np.zeros((1, 2)), np.array([(0, 0)]), T, lat,
                                        1e-8, 1e-13, 100000)
    assert s[0] == 0
    return v[0]


@pytest.mark.parametrize("tp", [-0.25, -0.35, -0.1])
def test_band_edges_and_van_hove_energy_fix_the_hopping_terms(tp):
    # ph_00(q = 0, T) = int -nF'(e) d^2k/(2pi)^2 is the density of states at the
    # Fermi level smeared over ~T.  Hand-derived features of the t-t' band,
    # independent of the oracle's formula, fix both hopping terms:
    #  * band bottom at k = 0: e ~ -4t - 4t' + (t + 2t') k^2, a 2-D step of
    #    height 1 / (4 pi (t + 2t')); at mu on the edge the smeared DOS is half
    #    the step;
    #  * band top at (pi, pi): e ~ 4t - 4t' - (t - 2t') k^2, half of
    #    1 / (4 pi (t - 2t'));
    #  * saddle points at (pi, 0), (0, pi): e = 4t' - mu, so the logarithmic
    #    van Hove peak of the DOS sits at mu = 4t'.
    # A wrong t' coefficient (say 2t' for 4t') moves the edges and the peak.
    t, T = 1.0, 0.004
    bottom = _ph00_q0(T, (t, tp, -4 * t - 4 * tp))
    top = _ph00_q0(T, (t, tp, 4 * t - 4 * tp))
    assert abs(bottom - 1.0 / (8 * math.pi * (t + 2 * tp))) < 0.02 * bottom
    assert abs(top - 1.0 / (8 * math.pi * (t - 2 * tp))) < 0.02 * top
    # well outside the band the smeared DOS vanishes
    assert _ph00_q0(T, (t, tp, -4 * t - 4 * tp - 0.2)) < 1e-6
    Tv = 0.02
    mus = 4 * tp + np.arange(-0.3, 0.3001, 0.01)
    dos = np.array([_ph00_q0(Tv, (t, tp, mu)) for mu in mus])
    peak = mus[int(np.argmax(dos))]
    assert abs(peak - 4 * tp) <= 0.04, peak
    assert dos.max() > 1.5 * min(dos[0], dos[-1])
