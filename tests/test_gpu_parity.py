"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Criterion, for integrals both sides report CONVERGED:
    |v_gpu - v_oracle| <= 2 max(rel_tol |v_oracle|, abs_tol) + 1e-12
(both results lie within their own error sums of the true integral, and each
error sum is below its tolerance).  For integrals either side stops on the
region budget, |v_gpu - v_oracle| <= E_gpu + E_oracle + 1e-12.
The error sum |Q_N - Q_2N| of Sec. 3 is an estimate, not a bound, so either
side can stop with an error larger than its estimate (a false convergence).
A pair that disagrees beyond the criterion is decided by the integral's
definition: a dense periodic trapezoid evaluation converged to 1e-13
(oracle.brute_force); the GPU result must lie within 2 tol of it.
The oracle uses the strict greedy order of Algorithm 1 and the GPU splits a
batch of regions per round, so the two partitions differ and the comparison
is at tolerance level, never bitwise.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1610_09991_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LAT = W.LATTICE


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def paid(torch):
    from paper_1610_09991_gb300 import build as B
    B.build()
    from paper_1610_09991_gb300 import paid as P
    return P


def _dev(torch, a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def run_gpu(paid, torch, ctx, batches):
    dbs = []
    for b in batches:
        dbs.append(dict(kind=b.kind, T=b.T, q=_dev(torch, b.q, torch.float64),
                        lm=_dev(torch, b.lm, torch.int32), rel_tol=b.rel_tol,
                        abs_tol=b.abs_tol, max_regions=b.max_regions))
    outs = ctx.integrate_multi(dbs)
    torch.cuda.synchronize()
    return [tuple(x.cpu().numpy() for x in (r.values, r.errors, r.regions, r.status)) for r in outs]


def assert_parity(g, o, rel, ab, ident=None, max_adjudicated=0.01):
    """ident(i) -> (kind, q, l, m, T) of integral i, for adjudication."""
    v, e, r, s = g
    vo, eo, ro, so = o
    assert np.all(np.isin(s, [0, 1, 2, 3, 4]))
    both = (s == 0) & (so == 0)
    d = np.abs(v - vo)
    tol1 = np.maximum(rel * np.abs(vo), ab)
    bad = both & (d > 2 * tol1 + 1e-12)
    rest = ~both & (s != 2) & (so != 2)
    bad |= rest & (d > e + eo + 1e-12)
    idx = np.where(bad)[0]
    assert ident is not None or idx.size == 0, (idx[:10], v[idx][:5], vo[idx][:5])
    assert idx.size <= max(1, max_adjudicated * len(v)), idx.size
    for i in idx:
        kind, q, l, m, T = ident(int(i))
        truth, M = oracle.brute_force(kind, q, l, m, T, LAT)
        assert np.isfinite(truth), (i, "brute force did not converge")
        t = max(rel * abs(truth), ab)
        assert abs(v[i] - truth) <= 2 * t + 1e-12, (i, v[i], vo[i], truth)
    # both sides agree on which integrals are non-finite
    assert np.array_equal(s == 2, so == 2)
    return both.sum()


def batch_ident(b):
    npairs = b.lm.shape[0]
    return lambda i: (b.kind, b.q[i // npairs], int(b.lm[i % npairs][0]),
                      int(b.lm[i % npairs][1]), b.T)


def flat_ident(flat, idx):
    return lambda i: (int(flat["kind"][idx[i]]), flat["q"][idx[i]], int(flat["lm"][idx[i]][0]),
                      int(flat["lm"][idx[i]][1]), float(flat["T"][idx[i]]))


def test_first_shell_batch_matches_oracle(paid, torch):
    w = W.config_first_shell()
    b = w.batches[0]
    ctx = paid.Context(*w.lattice, ffset=5)
    (g,) = run_gpu(paid, torch, ctx, [b])
    o = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol, b.max_regions)
    assert np.all(g[3] == 0) and np.all(o[3] == 0)
    assert assert_parity(g, o, b.rel_tol, b.abs_tol, batch_ident(b)) >= b.n - 1
    # each result within its own error estimate, and the budget respected
    assert np.all(g[1] <= np.maximum(b.abs_tol, b.rel_tol * np.abs(g[0])))
    assert np.all((g[2] - 16) % 3 == 0) and np.all(g[2] <= b.max_regions)
    st = ctx.last_stats()
    assert st["region_evals"] >= g[2].sum()


def test_flow_step_small_grid_matches_oracle(paid, torch):
    # the 93,312-integral flow-step batch on a 4 x 4 q grid: 2 x 16 x 81 integrals
    w = W.config_flow_step(T=0.05, nq=4)
    ctx = paid.Context(*w.lattice, ffset=9)
    gs = run_gpu(paid, torch, ctx, w.batches)
    for b, g in zip(w.batches, gs):
        o = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol,
                                   b.max_regions)
        n = assert_parity(g, o, b.rel_tol, b.abs_tol, batch_ident(b))
        assert n >= 0.9 * b.n


def test_full_flow_step_sampled(paid, torch):
    # 93,312 integrals at T = 0.05, checked on a seeded sample the oracle computes one by one
    w = W.config_flow_step()
    ctx = paid.Context(*w.lattice, ffset=9)
    gs = run_gpu(paid, torch, ctx, w.batches)
    g = tuple(np.concatenate([x[i] for x in gs]) for i in range(4))
    flat = W.flatten(w)
    idx = W.sample_indices(w.n, 240, seed=1234)
    o = oracle.integrate_list(flat["kind"][idx], flat["q"][idx], flat["lm"][idx],
                              flat["T"][idx], LAT, 1e-6, 1e-10, 100000)
    assert_parity(tuple(x[idx] for x in g), o, 1e-6, 1e-10, flat_ident(flat, idx))
    # properties at full size
    v, e, r, s = g
    assert np.all(np.isin(s, [0, 1]))
    conv = s == 0
    assert np.all(e[conv] <= np.maximum(1e-10, 1e-6 * np.abs(v[conv])))
    assert np.all(r <= 100000) and np.all((r - 16) % 3 == 0)
    # pp bubbles are symmetric in (l, m): I_lm = I_ml, within 2 tol
    vpp = v[w.batches[0].n:].reshape(576, 9, 9)
    tol = 2 * np.maximum(1e-6 * np.abs(vpp), 1e-10) + 1e-12
    assert np.all(np.abs(vpp - vpp.transpose(0, 2, 1)) <= tol + tol.transpose(0, 2, 1))


def test_monomials_exact(paid, torch):
    lm = np.array([(a, b) for a in range(0, 12) for b in range(0, 12)],
                  dtype=np.int32)
    b = W.Batch(W.MONOMIAL, 1.0, np.zeros((1, 2)), lm, 1e-10, 1e-14, 20000)
    ctx = paid.Context(*LAT, ffset=9, init_level=0)
    (g,) = run_gpu(paid, torch, ctx, [b])
    v, e, r, s = g
    for i, (a, c) in enumerate(lm):
        ex = 1.0 / ((a + 1) * (c + 1)) if (a % 2 == 0 and c % 2 == 0) else 0.0
        assert s[i] == 0
        assert abs(v[i] - ex) <= max(e[i], 1e-15) + 1e-15
        if a <= 5 and c <= 5:
            assert r[i] == 1


def test_overlap_gram_shift_matrix(paid, torch):
    from tests import np_ref
    q = np.array([(0.0, 0.0), (0.7, -1.9), (math.pi, math.pi)])
    b = W.Batch(W.OVERLAP, 1.0, q, W.all_pairs(9), 1e-12, 1e-12, 20000)
    ctx = paid.Context(*LAT, ffset=9, init_level=0)
    (g,) = run_gpu(paid, torch, ctx, [b])
    v = g[0].reshape(3, 9, 9)
    for i in range(3):
        assert np.allclose(v[i], np_ref.shift_matrix(q[i]).T, atol=2e-12)


def test_rule_n6_matches_oracle(paid, torch):
    b = W.Batch(W.PH, 0.2, W.q_grid_bz(2), W.all_pairs(5)[::3], 1e-7, 1e-10, 20000)
    ctx = paid.Context(*LAT, ffset=5, rule_n=6)
    (g,) = run_gpu(paid, torch, ctx, [b])
    o = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol, b.max_regions,
                               rule_n=6)
    assert assert_parity(g, o, b.rel_tol, b.abs_tol, batch_ident(b)) > 0


def test_edge_cases(paid, torch):
    ctx = paid.Context(*LAT, ffset=5)
    q = np.array([(0.3, 1.2)])
    # invalid pair index (9 is outside the 5-function set) and NaN temperature
    lm = np.array([(0, 0), (9, 1), (2, 2)], dtype=np.int32)
    (g,) = run_gpu(paid, torch, ctx, [W.Batch(W.PH, 0.5, q, lm)])
    assert list(g[3]) == [0, 2, 0]
    (g,) = run_gpu(paid, torch, ctx, [W.Batch(W.PH, float("nan"), q, lm[:1])])
    assert g[3][0] == 2
    # tiny budget: the same leaf-count cap as the oracle
    (g,) = run_gpu(paid, torch, ctx, [W.Batch(W.PH, 0.01, q, np.array([(1, 2)]), 1e-12, 1e-16, 100)])
    assert g[3][0] == 1 and 97 < g[2][0] <= 100
    # a single region: L0 = 0, a monomial the coarse rule integrates exactly
    c0 = paid.Context(*LAT, ffset=5, init_level=0)
    (g,) = run_gpu(paid, torch, c0, [W.Batch(W.MONOMIAL, 1.0, np.zeros((1, 2)), np.array([(2, 4)]))])
    assert g[2][0] == 1 and abs(g[0][0] - 1.0 / 15.0) < 1e-15
    # empty batch
    out = ctx.integrate_multi([dict(kind=0, T=0.5, q=torch.zeros((0, 2), dtype=torch.float64,
                                                                   device="cuda"),
                                    lm=torch.zeros((1, 2), dtype=torch.int32, device="cuda"))])
    assert out[0].values.numel() == 0


def test_round_cap_and_pool_full(paid, torch):
    b = W.Batch(W.PH, 0.05, W.q_grid_bz(2), W.all_pairs(5), 1e-8, 1e-12, 100000)
    ctx = paid.Context(*LAT, ffset=5, max_rounds=1)
    (g,) = run_gpu(paid, torch, ctx, [b])
    assert ctx.last_rc == paid.ERR_TIMEOUT
    assert np.all(np.isin(g[3], [0, 3])) and np.any(g[3] == 3)
    # a pool that holds the initial partition and little more
    ctx2 = paid.Context(*LAT, ffset=5)
    dbs = [dict(kind=b.kind, T=b.T, q=_dev(torch, b.q, torch.float64),
                lm=_dev(torch, b.lm, torch.int32), rel_tol=b.rel_tol, abs_tol=b.abs_tol,
                max_regions=b.max_regions)]
    (r,) = ctx2.integrate_multi(dbs, pool_capacity=b.n * 16 + 64)
    assert ctx2.last_rc == paid.ERR_POOL
    st = r.status.cpu().numpy()
    assert np.all(np.isin(st, [0, 1, 4])) and np.any(st == 4)
    # the default policy grows the pool and finishes (converged or on the budget)
    (g,) = run_gpu(paid, torch, ctx2, [b])
    assert ctx2.last_rc == paid.OK
    assert np.all(np.isin(g[3], [0, 1])) and np.any(g[3] == 0)


def test_bitwise_reproducible(paid, torch):
    w = W.config_flow_step(T=0.1, nq=2)
    ctx = paid.Context(*w.lattice, ffset=9)
    a = run_gpu(paid, torch, ctx, w.batches)
    b = run_gpu(paid, torch, ctx, w.batches)
    for x, y in zip(a, b):
        for u, v in zip(x, y):
            assert np.array_equal(u, v)


def test_host_entry_point(paid, torch):
    w = W.config_first_shell()
    b = w.batches[0]
    ctx = paid.Context(*w.lattice, ffset=5)
    (r,), h2d, d2h = ctx.integrate_host([dict(kind=b.kind, T=b.T, q=b.q, lm=b.lm)])
    assert h2d == b.q.nbytes + b.lm.astype(np.int32).nbytes
    assert d2h == b.n * (8 + 8 + 8 + 4)
    (g,) = run_gpu(paid, torch, ctx, [b])
    assert np.array_equal(r.values, g[0])


def test_streaming_pool_smaller_than_the_batch(paid, torch):
    # a pool that holds ~1/3 of the batch's final regions: integrals enter as
    # room frees up and splits are throttled, with the same results
    b = W.Batch(W.PH, 0.2, W.q_grid_bz(4), W.all_pairs(9)[::5], 1e-6, 1e-10, 100000)
    ctx = paid.Context(*LAT, ffset=9)
    (g,) = run_gpu(paid, torch, ctx, [b])
    full = ctx.last_stats()
    dbs = [dict(kind=b.kind, T=b.T, q=_dev(torch, b.q, torch.float64),
                lm=_dev(torch, b.lm, torch.int32), rel_tol=b.rel_tol, abs_tol=b.abs_tol,
                max_regions=b.max_regions)]
    (r,) = ctx.integrate_multi(dbs, pool_capacity=max(full["peak_pool"] // 3, 20000))
    torch.cuda.synchronize()
    st = ctx.last_stats()
    assert ctx.last_rc == paid.OK
    assert st["throttled_rounds"] > 0 or st["rounds"] > full["rounds"]
    assert np.array_equal(r.status.cpu().numpy(), g[3])
    v = r.values.cpu().numpy()
    tol = np.maximum(1e-6 * np.abs(g[0]), 1e-10)
    assert np.all(np.abs(v - g[0]) <= 2 * tol + 1e-12)


def test_temperature_sweep_sampled(paid, torch):
    # 12 temperatures from 1 down to 0.005 x 4x4 zone grid x 81 pairs x {ph, pp}
    # (31,104 integrals of very uneven depth) in one FP64 call, against the
    # oracle on a seeded sample
    w = W.config_temperature_sweep(nq=4)
    ctx = paid.Context(*w.lattice, ffset=9)
    gs = run_gpu(paid, torch, ctx, w.batches)
    g = tuple(np.concatenate([x[i] for x in gs]) for i in range(4))
    flat = W.flatten(w)
    idx = W.sample_indices(w.n, 48, seed=77)
    o = oracle.integrate_list(flat["kind"][idx], flat["q"][idx], flat["lm"][idx],
                              flat["T"][idx], LAT, 1e-6, 1e-10, 100000)
    assert_parity(tuple(x[idx] for x in g), o, 1e-6, 1e-10, flat_ident(flat, idx))
    assert np.all(np.isin(g[3], [0, 1]))
    # deeper at low T: mean region count grows as T falls
    r = g[2].reshape(12, -1).mean(axis=1)
    assert r[-1] > 5 * r[0]
