"""Pins of the oracle's group driver: Algorithm 2 with the global error of
Sec. 4 (one heap and one error sum over all (l, m) pairs of a (kind, q)).

* A group of one pair is Algorithm 1: the result must equal the per-integral
  driver's bit for bit (that driver is pinned in test_oracle_driver.py).
* A hand-stepped group greedy written here with heapq and the numpy rule of
  test_oracle_driver.py must reproduce every pair's value, error and leaf
  count on tiny budgets.
* Values against the definition: at T = 0.5 the pairs' values are compared
  with the dense periodic trapezoid, and their summed deviation must lie
  within the group tolerance.
* The stopping test is the group's, not each pair's: the sum of the pairs'
  errors meets the group tolerance while a pair that vanishes by symmetry
  keeps an error far above the per-integral absolute floor.
"""
import heapq

import numpy as np
import pytest

import oracle
from tests.test_oracle_driver import _region

LAT = (1.0, -0.25, -1.0)


def _group_greedy(kind, q, pairs, T, L0, rel, ab, budget):
    heap = []
    leaves = [0] * len(pairs)
    for c, (l, m) in enumerate(pairs):
        for ix in range(2 ** L0):
            for iy in range(2 ** L0):
                a, b = _region(kind, q, l, m, T, L0, ix, iy)
                heapq.heappush(heap, (-abs(a - b), c, L0, ix, iy, b))
                leaves[c] += 1
    while True:
        V = [sum(t[5] for t in heap if t[1] == c) for c in range(len(pairs))]
        E = [sum(-t[0] for t in heap if t[1] == c) for c in range(len(pairs))]
        if sum(E) <= max(ab, rel * sum(abs(v) for v in V)):
            return V, E, leaves, 0
        _, c, L, ix, iy, _ = heap[0]
        if leaves[c] + 3 > budget:
            return V, E, leaves, 1
        heapq.heappop(heap)
        l, m = pairs[c]
        for da in (0, 1):
            for db in (0, 1):
                a, b = _region(kind, q, l, m, T, L + 1, 2 * ix + da, 2 * iy + db)
                heapq.heappush(heap, (-abs(a - b), c, L + 1, 2 * ix + da, 2 * iy + db, b))
        leaves[c] += 3


@pytest.mark.parametrize("kind,q,pairs,T,L0,rel,budget", [
    (0, (0.31, 1.13), [(0, 0), (1, 3), (4, 4)], 0.2, 1, 1e-12, 16),
    (1, (-0.7, 2.4), [(4, 2), (2, 4), (0, 8)], 0.1, 1, 1e-12, 22),
    (0, (2.2, -0.9), [(5, 7), (1, 1)], 0.3, 2, 1e-4, 40),
])
def test_group_oracle_matches_hand_stepped_greedy(kind, q, pairs, T, L0, rel, budget):
    V, E, leaves, st = _group_greedy(kind, q, pairs, T, L0, rel, 1e-16, budget)
    v, e, r, s = oracle.integrate_group_global(kind, np.array([q]), np.array(pairs), T, LAT,
                                               rel, 1e-16, budget, init_level=L0)
    assert np.all(s == st)
    assert r.tolist() == leaves
    scale = max(1.0, max(abs(x) for x in V))
    assert np.allclose(v, V, rtol=0, atol=1e-13 * scale)
    assert np.allclose(e, E, rtol=0, atol=1e-13 * scale)


def test_ties_go_to_the_smaller_pair_index():
    # two copies of one pair tie at every region; the group stops between the
    # copies' splits, so the first copy ends with one split more
    q, pairs = (0.31, 1.13), [(1, 3), (1, 3)]
    V, E, leaves, st = _group_greedy(0, q, pairs, 0.2, 1, 3e-3, 1e-16, 1000)
    v, e, r, s = oracle.integrate_group_global(0, np.array([q]), np.array(pairs), 0.2, LAT,
                                               3e-3, 1e-16, 1000, init_level=1)
    assert st == 0 and np.all(s == 0)
    assert r.tolist() == leaves and leaves[0] == leaves[1] + 3
    assert np.allclose(e, E, rtol=0, atol=1e-15)


@pytest.mark.parametrize("kind,q,lm,T", [
    (0, (0.4, 1.7), (1, 2), 0.1),
    (1, (2.9, -0.3), (3, 3), 0.05),
    (4, (1.2, 0.6), (0, 4), 0.2),      # flow kind: T is the regulator scale Omega
])
def test_one_pair_group_is_algorithm_1(kind, q, lm, T):
    q = np.array([q])
    lm = np.array([lm], dtype=np.int32)
    a = oracle.integrate_group_global(kind, q, lm, T, LAT, 1e-6, 1e-10, 100000)
    b = oracle.integrate_batch(kind, q, lm, T, LAT, 1e-6, 1e-10, 100000)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_group_values_against_the_definition():
    q = np.array([(0.7, 1.9)])
    pairs = np.array([(0, 0), (1, 1), (1, 2), (2, 4), (3, 0), (4, 4)], dtype=np.int32)
    rel = 1e-8
    v, e, r, s = oracle.integrate_group_global(0, q, pairs, 0.5, LAT, rel, 0.0, 100000)
    assert np.all(s == oracle.CONVERGED)
    tol = rel * np.abs(v).sum()
    assert e.sum() <= tol
    truth = np.array([oracle.brute_force(0, q[0], int(l), int(m), 0.5, LAT)[0] for l, m in pairs])
    assert np.abs(v - truth).sum() <= tol


def test_the_stopping_test_is_the_groups():
    # q on the kx axis: f_4 = sqrt2 sin ky is odd under ky -> -ky and f_0 even,
    # and the bubble is even in ky there, so the pair (0, 4) vanishes
    q = np.array([(1.3, 0.0)])
    pairs = np.array([(0, 0), (1, 1), (0, 4)], dtype=np.int32)
    rel = 1e-7
    v, e, r, s = oracle.integrate_group_global(0, q, pairs, 0.1, LAT, rel, 1e-10, 100000)
    assert np.all(s == oracle.CONVERGED)
    assert e.sum() <= rel * np.abs(v).sum()
    assert abs(v[2]) < 1e-12
    assert e[2] > 1e-10            # a per-pair test would have refined it further
    # the per-integral driver at the same tolerances holds the vanishing pair
    # to the absolute floor and needs more leaves for it
    vi, ei, ri, si = oracle.integrate_batch(0, q, pairs, 0.1, LAT, rel, 1e-10, 100000)
    assert ei[2] <= 1e-10 and ri[2] > r[2]


def test_paper_absolute_criterion_and_independent_groups():
    qs = np.array([(0.3, 0.9), (2.5, 2.5), (-1.0, 0.2)])
    pairs = np.array([(0, 0), (2, 1), (3, 3)], dtype=np.int32)
    eps = 1e-9
    v, e, r, s = oracle.integrate_group_global(1, qs, pairs, 0.2, LAT, 0.0, eps, 100000)
    assert np.all(s == oracle.CONVERGED)
    for i in range(3):
        assert e[3 * i:3 * i + 3].sum() <= eps
        one = oracle.integrate_group_global(1, qs[i:i + 1], pairs, 0.2, LAT, 0.0, eps, 100000)
        for x, y in zip(one, (v, e, r, s)):
            assert np.array_equal(x, y[3 * i:3 * i + 3])


def test_group_budget_and_nonfinite():
    q = np.array([(0.5, 0.5)])
    pairs = np.array([(1, 2), (0, 0)], dtype=np.int32)
    v, e, r, s = oracle.integrate_group_global(0, q, pairs, 0.01, LAT, 1e-12, 1e-16, 40)
    assert np.all(s == oracle.BUDGET) and r.max() <= 40 and r.max() > 37
    v, e, r, s = oracle.integrate_group_global(0, q, pairs, float("nan"), LAT, 1e-6, 1e-10, 1000)
    assert np.all(s == oracle.NONFINITE)
    with pytest.raises(ValueError):
        oracle.integrate_group_global(0, q, np.zeros((0, 2), np.int32), 0.1, LAT, 1e-6, 1e-10, 100)
