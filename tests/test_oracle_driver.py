"""Pins of the oracle's adaptive driver (Algorithm 1 with the 4-way split of
Algorithm 2, Listings 1-5 for one integral).

A hand-stepped greedy written here with heapq and a numpy tensor CC rule (own
weights from the moment equations) must reproduce the oracle's leaf set and
value exactly on tiny budgets; budget exhaustion and non-finite parameters
give their statuses.
"""
import heapq
import math

import numpy as np
import pytest

import oracle
from tests import np_ref

LAT = (1.0, -0.25, -1.0)


def _cc(N):
    x = np.cos(np.arange(N + 1) * math.pi / N)
    V = np.vstack([np.polynomial.chebyshev.chebval(x, np.eye(N + 1)[k]) for k in range(N + 1)])
    mu = np.array([2.0 / (1 - k * k) if k % 2 == 0 else 0.0 for k in range(N + 1)])
    return x, np.linalg.solve(V, mu)


def _region(kind, q, l, m, T, L, ix, iy, N=4):
    xf, wf = _cc(2 * N)
    _, wc = _cc(N)
    h = 2 * math.pi / 2 ** L
    kx = -math.pi + ix * h + 0.5 * h * (1 + xf)
    ky = -math.pi + iy * h + 0.5 * h * (1 + xf)
    KX, KY = np.meshgrid(kx, ky, indexing="ij")
    g = np_ref.integrand(kind, q, l, m, T, LAT, KX, KY)
    q2 = 0.25 * h * h * float(wf @ g @ wf)
    q1 = 0.25 * h * h * float(wc @ g[::2, ::2] @ wc)
    return q1, q2


def _greedy(kind, q, l, m, T, L0, rel, ab, budget):
    heap = []
    for ix in range(2 ** L0):
        for iy in range(2 ** L0):
            a, b = _region(kind, q, l, m, T, L0, ix, iy)
            heapq.heappush(heap, (-abs(a - b), L0, ix, iy, b))
    while True:
        V = sum(t[4] for t in heap)
        E = sum(-t[0] for t in heap)
        if E <= max(ab, rel * abs(V)):
            return V, E, heap, 0
        if len(heap) + 3 > budget:
            return V, E, heap, 1
        _, L, ix, iy, _ = heapq.heappop(heap)
        for da in (0, 1):
            for db in (0, 1):
                a, b = _region(kind, q, l, m, T, L + 1, 2 * ix + da, 2 * iy + db)
                heapq.heappush(heap, (-abs(a - b), L + 1, 2 * ix + da, 2 * iy + db, b))


@pytest.mark.parametrize("kind,q,l,m,T,L0,budget", [
    (0, (0.31, 1.13), 1, 3, 0.2, 1, 16),
    (1, (-0.7, 2.4), 4, 2, 0.1, 2, 34),
    (0, (2.2, -0.9), 5, 7, 0.05, 2, 40),
    (1, (1.9, 0.3), 0, 8, 0.3, 0, 13),
])
def test_oracle_matches_hand_stepped_greedy(kind, q, l, m, T, L0, budget):
    V, E, heap, st = _greedy(kind, q, l, m, T, L0, 1e-12, 1e-16, budget)
    res = oracle.integrate_trace(kind, q, l, m, T, LAT, 1e-12, 1e-16, budget, init_level=L0)
    assert res["status"] == st
    assert res["regions"] == len(heap)
    mine = sorted((t[1], t[2], t[3]) for t in heap)
    theirs = sorted(zip(res["level"].tolist(), res["ix"].tolist(), res["iy"].tolist()))
    assert mine == theirs
    assert abs(res["value"] - V) < 1e-13 * max(1.0, abs(V))
    assert abs(res["error"] - E) < 1e-13 * max(1.0, abs(E))
    # leaf value sum is the returned value (Listing 5)
    assert abs(res["val2N"].sum() - res["value"]) < 1e-15 * max(1.0, abs(V)) + 1e-18


def test_budget_status_and_cap():
    q = np.array([(0.5, 0.5)])
    lm = np.array([(1, 2)], dtype=np.int32)
    v, e, r, s = oracle.integrate_batch(0, q, lm, 0.01, LAT, 1e-12, 1e-16, 16, init_level=2)
    assert s[0] == oracle.BUDGET and r[0] == 16
    v, e, r, s = oracle.integrate_batch(0, q, lm, 0.01, LAT, 1e-12, 1e-16, 100, init_level=2)
    assert s[0] == oracle.BUDGET and r[0] <= 100 and r[0] > 97


def test_nonfinite_parameters():
    q = np.array([(0.5, 0.5)])
    lm = np.array([(0, 0)], dtype=np.int32)
    v, e, r, s = oracle.integrate_batch(0, q, lm, float("nan"), LAT, 1e-6, 1e-10, 1000)
    assert s[0] == oracle.NONFINITE
    v, e, r, s = oracle.integrate_batch(0, np.array([(float("inf"), 0.0)]), lm, 0.5, LAT,
                                        1e-6, 1e-10, 1000)
    assert s[0] == oracle.NONFINITE


def test_empty_batch():
    v, e, r, s = oracle.integrate_batch(0, np.zeros((0, 2)), np.array([(0, 0)]), 0.5, LAT,
                                        1e-6, 1e-10, 1000)
    assert v.shape == (0,)
