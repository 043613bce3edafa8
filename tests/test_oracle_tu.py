"""Pins of the oracle's truncated-unity products (Eqs. matmul-P/C/D, Sec. 2):
explicit index loops on small cases, and the closed forms for unit couplings."""
import numpy as np

import oracle


def _loops(VP, VC, VD, Xpp, Xph):
    nq, n, _ = VP.shape
    dP = np.zeros_like(VP)
    dC = np.zeros_like(VP)
    dD = np.zeros_like(VP)
    for k in range(nq):
        for a in range(n):
            for b in range(n):
                sp = sc = sd = 0.0
                for i in range(n):
                    for j in range(n):
                        sp += VP[k, a, i] * Xpp[k, i, j] * VP[k, j, b]
                        sc -= VC[k, a, i] * Xph[k, i, j] * VC[k, j, b]
                        sd += (2.0 * VD[k, a, i] * Xph[k, i, j] * VD[k, j, b]
                               - VC[k, a, i] * Xph[k, i, j] * VD[k, j, b]
                               - VD[k, a, i] * Xph[k, i, j] * VC[k, j, b])
                dP[k, a, b], dC[k, a, b], dD[k, a, b] = sp, sc, sd
    return dP, dC, dD


def test_products_match_index_loops():
    rng = np.random.default_rng(5)
    for n in (1, 5, 9):
        m = [rng.normal(size=(3, n, n)) for _ in range(5)]
        got = oracle.tu_flow_rhs(*m)
        want = _loops(*m)
        for g, w in zip(got, want):
            assert np.allclose(g, w, rtol=1e-13, atol=1e-13)


def test_unit_couplings():
    rng = np.random.default_rng(6)
    X1, X2 = rng.normal(size=(2, 4, 9, 9))
    eye = np.broadcast_to(np.eye(9), (4, 9, 9))
    dP, dC, dD = oracle.tu_flow_rhs(eye, eye, eye, X1, X2)
    assert np.array_equal(dP, X1) and np.array_equal(dC, -X2)
    assert np.allclose(dD, 0.0, atol=1e-15)       # 2 X - X - X
    # V^C = 0: only the direct term of dD survives
    zero = np.zeros((4, 9, 9))
    dP, dC, dD = oracle.tu_flow_rhs(eye, zero, eye, X1, X2)
    assert np.array_equal(dC, zero) and np.allclose(dD, 2 * X2)
