"""Shared-partition (group) mode against the FP64 oracle.

Region level: the group kernel's Q_N and Q_2N of every pair on a region,
computed from separable moments, against the oracle's direct nested rule on
the same region (Sec. 3), pair by pair.  The two sum the same nodes in a
different order, so they agree to rounding.

Integral level: every integral of a group meets its own tolerance on the
group's shared partition, so the group results satisfy the same parity
criterion against the per-integral oracle as the per-integral mode
(test_gpu_parity.py): 2 max(rel_tol |v|, abs_tol) + 1e-12, disagreements
decided by the converged brute-force trapezoid.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1610_09991_gb300 import workloads as W
from tests.test_gpu_parity import assert_parity, batch_ident, flat_ident

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


def _run(paid, torch, ctx, batches, pool_capacity=None):
    dbs = [dict(kind=b.kind, T=b.T, q=_dev(torch, b.q, torch.float64),
                lm=_dev(torch, b.lm, torch.int32), rel_tol=b.rel_tol, abs_tol=b.abs_tol,
                max_regions=b.max_regions) for b in batches]
    outs = ctx.integrate_multi(dbs, pool_capacity=pool_capacity)
    torch.cuda.synchronize()
    return [tuple(x.cpu().numpy() for x in (r.values, r.errors, r.regions, r.status)) for r in outs]


@pytest.mark.parametrize("kind,T", [(W.PH, 0.05), (W.PP, 0.05), (W.PH, 0.7), (W.OVERLAP, 1.0)])
def test_rule_regions_match_the_oracle_rule(paid, torch, kind, T):
    rng = np.random.default_rng(17 + kind)
    ctx = paid.Context(*LAT, ffset=9)
    lm = W.all_pairs(9)
    regs = [(0, 0, 0), (1, 1, 0), (2, 3, 1)]
    for L in (3, 5, 8, 12, 20, 29):
        for _ in range(3):
            regs.append((L, int(rng.integers(0, 2 ** L)), int(rng.integers(0, 2 ** L))))
    regs.append((30, 0, 0))       # invalid level
    regs.append((2, 4, 0))        # index outside 2^level
    regions = np.array(regs, dtype=np.int32)
    for q in (np.array([0.3, -2.1]), np.array([math.pi, 0.0])):
        q2, dq = ctx.rule_regions(kind, _dev(torch, q, torch.float64), _dev(torch, lm, torch.int32),
                                  T, _dev(torch, regions, torch.int32))
        q2, dq = q2.cpu().numpy(), dq.cpu().numpy()
        assert np.all(np.isnan(q2[-2:])) and np.all(np.isnan(dq[-2:]))
        for r, (L, ix, iy) in enumerate(regs[:-2]):
            ref = np.array([oracle.region_eval(kind, q, int(l), int(m), T, LAT, L, ix, iy)
                            for l, m in lm])          # (Q_N, Q_2N) per pair
            scale = np.abs(ref).max() + 1e-300
            assert np.all(np.abs(q2[r] - ref[:, 1]) <= 1e-12 * scale), (L, ix, iy)
            assert np.all(np.abs(dq[r] - (ref[:, 0] - ref[:, 1])) <= 1e-12 * scale), (L, ix, iy)


@pytest.mark.parametrize("N", [6, 8, 10, 12])
def test_rule_regions_higher_order(paid, torch, N):
    ctx = paid.Context(*LAT, ffset=9, rule_n=N, group_mode=1)
    lm = W.all_pairs(9)[::4]
    q = np.array([1.1, 0.4])
    regs = np.array([(0, 0, 0), (4, 3, 9), (11, 1000, 17)], dtype=np.int32)
    q2, dq = ctx.rule_regions(W.PP, _dev(torch, q, torch.float64), _dev(torch, lm, torch.int32),
                              0.1, _dev(torch, regs, torch.int32))
    q2, dq = q2.cpu().numpy(), dq.cpu().numpy()
    for r, (L, ix, iy) in enumerate(regs):
        ref = np.array([oracle.region_eval(W.PP, q, int(l), int(m), 0.1, LAT, int(L), int(ix),
                                           int(iy), rule_n=N) for l, m in lm])
        scale = np.abs(ref).max() + 1e-300
        assert np.all(np.abs(q2[r] - ref[:, 1]) <= 1e-12 * scale)
        assert np.all(np.abs(dq[r] - (ref[:, 0] - ref[:, 1])) <= 1e-12 * scale)


def test_group_first_shell_matches_oracle(paid, torch):
    w = W.config_first_shell()
    b = w.batches[0]
    ctx = paid.Context(*w.lattice, ffset=5, group_mode=1)
    (g,) = _run(paid, torch, ctx, [b])
    o = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol, b.max_regions)
    assert np.all(g[3] == 0)
    assert assert_parity(g, o, b.rel_tol, b.abs_tol, batch_ident(b)) >= b.n - 1
    # every integral within its own tolerance; one region count per group
    assert np.all(g[1] <= np.maximum(b.abs_tol, b.rel_tol * np.abs(g[0])))
    r = g[2].reshape(16, 25)
    assert np.all(r == r[:, :1]) and np.all((r - 16) % 3 == 0)
    st = ctx.last_stats()
    assert st["region_evals"] >= r[:, 0].sum()


@pytest.mark.parametrize("T", [0.05, 0.5])
def test_group_flow_step_small_grid_matches_oracle(paid, torch, T):
    w = W.config_flow_step(T=T, nq=4)
    ctx = paid.Context(*w.lattice, ffset=9, group_mode=1)
    gs = _run(paid, torch, ctx, w.batches)
    for b, g in zip(w.batches, gs):
        assert np.all(np.isin(g[3], [0, 1]))
        o = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol,
                                   b.max_regions)
        n = assert_parity(g, o, b.rel_tol, b.abs_tol, batch_ident(b))
        assert n >= 0.9 * b.n


def test_group_full_flow_step_sampled(paid, torch):
    # all 93,312 integrals of the flow step in 1152 groups, checked on a seeded
    # sample that the oracle computes one by one, and by the pp symmetry
    w = W.config_flow_step()
    ctx = paid.Context(*w.lattice, ffset=9, group_mode=1)
    gs = _run(paid, torch, ctx, w.batches)
    g = tuple(np.concatenate([x[i] for x in gs]) for i in range(4))
    flat = W.flatten(w)
    idx = W.sample_indices(w.n, 240, seed=1234)
    o = oracle.integrate_list(flat["kind"][idx], flat["q"][idx], flat["lm"][idx],
                              flat["T"][idx], LAT, 1e-6, 1e-10, 100000)
    assert_parity(tuple(x[idx] for x in g), o, 1e-6, 1e-10, flat_ident(flat, idx))
    v, e, r, s = g
    assert np.all(np.isin(s, [0, 1]))
    conv = s == 0
    assert np.all(e[conv] <= np.maximum(1e-10, 1e-6 * np.abs(v[conv])))
    vpp = v[w.batches[0].n:].reshape(576, 9, 9)
    tol = 2 * np.maximum(1e-6 * np.abs(vpp), 1e-10) + 1e-12
    assert np.all(np.abs(vpp - vpp.transpose(0, 2, 1)) <= tol + tol.transpose(0, 2, 1))


def test_group_device_loop_matches_host_loop(paid, torch):
    w = W.config_flow_step(T=0.1, nq=2)
    a = _run(paid, torch, paid.Context(*LAT, ffset=9, group_mode=1, device_loop=1), w.batches)
    b = _run(paid, torch, paid.Context(*LAT, ffset=9, group_mode=1, device_loop=0), w.batches)
    for x, y in zip(a, b):
        for u, v in zip(x, y):
            assert np.array_equal(u, v)


def test_group_streaming_small_pool(paid, torch):
    b = W.Batch(W.PH, 0.2, W.q_grid_bz(4), W.all_pairs(9)[::5], 1e-6, 1e-10, 100000)
    ctx = paid.Context(*LAT, ffset=9, group_mode=1)
    (full,) = _run(paid, torch, ctx, [b])
    peak = ctx.last_stats()["peak_pool"]
    # room for half the batch's peak and at least four of its largest groups:
    # admitted groups grow ~30x from their 16-region start, and the first
    # group's round must fit beside the others for the pool to progress
    cap = max(peak // 2, 4 * int(full[2].max()))
    assert cap < peak
    (g,) = _run(paid, torch, ctx, [b], pool_capacity=cap)
    st = ctx.last_stats()
    assert ctx.last_rc == paid.OK and st["peak_pool"] <= cap < peak
    assert np.array_equal(g[3], full[3])
    tol = np.maximum(1e-6 * np.abs(full[0]), 1e-10)
    assert np.all(np.abs(g[0] - full[0]) <= 2 * tol + 1e-12)


def test_group_edge_cases(paid, torch):
    ctx = paid.Context(*LAT, ffset=5, group_mode=1)
    q = np.array([(0.3, 1.2), (-2.0, 0.5)])
    lm = np.array([(0, 0), (9, 1), (2, 2)], dtype=np.int32)      # (9, 1) is invalid
    (g,) = _run(paid, torch, ctx, [W.Batch(W.PH, 0.5, q, lm)])
    assert list(g[3]) == [0, 2, 0, 0, 2, 0] and np.isnan(g[0][1])
    (g,) = _run(paid, torch, ctx, [W.Batch(W.PH, float("nan"), q[:1], lm[:1])])
    assert g[3][0] == 2
    # tiny budget: the group stops at <= max_regions, pairs that met their
    # tolerance report CONVERGED, the others BUDGET
    (g,) = _run(paid, torch, ctx, [W.Batch(W.PH, 0.01, q[:1], np.array([(1, 2), (0, 0)]),
                                           1e-12, 1e-16, 100)])
    assert np.all(np.isin(g[3], [0, 1])) and np.any(g[3] == 1) and np.all(g[2] <= 100)
    # the monomial kind has no form-factor structure: refused in group mode
    with pytest.raises(paid.PaidError):
        _run(paid, torch, ctx, [W.Batch(W.MONOMIAL, 1.0, np.zeros((1, 2)), np.array([(2, 4)]))])


def test_group_static_entry(paid, torch):
    b = W.Batch(W.PP, 0.5, W.q_grid_bz(2), W.all_pairs(9), 1e-6, 1e-10, 20000)
    ctx = paid.Context(*LAT, ffset=9, group_mode=1)
    (g,) = _run(paid, torch, ctx, [b])
    r = ctx.integrate_batch_static(b.kind, _dev(torch, b.q, torch.float64),
                                   _dev(torch, b.lm, torch.int32), b.T, b.rel_tol, b.abs_tol,
                                   b.max_regions)
    torch.cuda.synchronize()
    assert np.array_equal(r.values.cpu().numpy(), g[0])
    assert np.array_equal(r.status.cpu().numpy(), g[3])


def test_own_exp_and_division_error_bounds(paid, torch):
    # the group kernel's exp(-x) (Tang's table-driven method) and division
    # (approximate reciprocal + Newton-Raphson) against correctly rounded
    # references: at most 2 ulp, and the flush-to-zero / NaN behaviour
    ctx = paid.Context(*LAT, ffset=9)
    rng = np.random.default_rng(3)
    x = np.concatenate([np.array([0.0, 1e-300, 1e-17, 5e-3, math.log(2) / 128, 1.0, 20.0,
                                  700.0, 707.5, 745.2, 800.0, 1e6]),
                        rng.uniform(0, 1, 20000), rng.uniform(0, 50, 20000),
                        rng.uniform(0, 708, 20000), np.exp(rng.uniform(-40, 6, 20000))])
    got = ctx.check_math(0, _dev(torch, x, torch.float64)).cpu().numpy()
    ref = np.exp(-x)
    normal = ref >= 2.0 ** -1022
    ulp = np.spacing(ref[normal])
    assert np.all(np.abs(got[normal] - ref[normal]) <= 2 * ulp)
    assert np.all(got[~normal] <= 2.0 ** -1021)
    nan = ctx.check_math(0, _dev(torch, np.array([np.nan]), torch.float64)).cpu().numpy()
    assert np.isnan(nan[0])
    a = rng.normal(size=40000) * np.exp(rng.uniform(-20, 20, 40000))
    b = rng.choice([-1.0, 1.0], 40000) * np.exp(rng.uniform(-30, 30, 40000))
    got = ctx.check_math(1, _dev(torch, a, torch.float64), _dev(torch, b, torch.float64))
    ref = a / b
    assert np.all(np.abs(got.cpu().numpy() - ref) <= 2 * np.spacing(np.abs(ref)))


def test_autotune_picks_a_candidate_and_caches_it(paid, torch, tmp_path):
    w = W.config_flow_step(T=0.05, nq=4)
    dbs = [dict(kind=b.kind, T=b.T, q=_dev(torch, b.q, torch.float64),
                lm=_dev(torch, b.lm, torch.int32), rel_tol=b.rel_tol, abs_tol=b.abs_tol,
                max_regions=b.max_regions) for b in w.batches]
    path = str(tmp_path / "tune.jsonl")
    ctx = paid.Context(*LAT, ffset=9, group_mode=1)
    o = ctx.autotune(dbs, path)
    assert o.cover in (0.5, 0.75, 0.9, 1.0) and o.eval_blocks in (608, 1216, 4864, 19456)
    assert o.rule_n in (4, 6, 8, 10, 12) and o.init_level in (2, 3)
    lines = open(path).read().splitlines()
    assert len(lines) == 1 and "group_mode=1" in lines[0] and '"init_level": ' in lines[0]
    # a second context applies the cached choice without a sample
    c2 = paid.Context(*LAT, ffset=9, group_mode=1)
    o2 = c2.autotune(None, path)
    assert ((o2.rule_n, o2.cover, o2.eval_blocks, o2.init_level)
            == (o.rule_n, o.cover, o.eval_blocks, o.init_level))
    # tuned options keep parity with the oracle on the sample
    gs = _run(paid, torch, ctx, w.batches)
    for b, g in zip(w.batches, gs):
        o_ = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol,
                                    b.max_regions, rule_n=o.rule_n, init_level=o.init_level)
        assert assert_parity(g, o_, b.rel_tol, b.abs_tol, batch_ident(b)) >= 0.9 * b.n
    # a per-integral context keeps its own entry (another key)
    c3 = paid.Context(*LAT, ffset=9)
    c3.autotune(dbs[:1], path)
    assert len(open(path).read().splitlines()) == 2


@pytest.mark.parametrize("N", [6, 8, 10, 12])
def test_group_higher_order_flow_step_matches_oracle(paid, torch, N):
    # the paper's best-performing rule (N = 6: 7 x 7 inside 13 x 13) and N = 8
    # (9 x 9 inside 17 x 17) in group mode, against the oracle with the same
    # rule and with the N = 4 rule
    w = W.config_flow_step(T=0.05, nq=4)
    ctx = paid.Context(*w.lattice, ffset=9, group_mode=1, rule_n=N, cover=1.0)
    gs = _run(paid, torch, ctx, w.batches)
    for b, g in zip(w.batches, gs):
        assert np.all(np.isin(g[3], [0, 1]))
        for rn in (N, 4):
            o = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol,
                                       b.max_regions, rule_n=rn)
            assert assert_parity(g, o, b.rel_tol, b.abs_tol, batch_ident(b)) >= 0.9 * b.n


@pytest.mark.parametrize("eval_fp32", [0, 1])
def test_group_temperature_sweep_in_one_call(paid, torch, eval_fp32):
    # the batching workload's recipe on a 4 x 4 q grid: 12 temperatures from 1
    # to 0.005 x {ph, pp} x 81 pairs = 31,104 integrals of very uneven depth in
    # one call (24 batches in one pool), shared partitions at N = 12; a seeded
    # oracle sample across all temperatures, one by one
    w = W.config_temperature_sweep(nq=4)
    ctx = paid.Context(*w.lattice, ffset=9, group_mode=1, rule_n=12, cover=1.0,
                       eval_fp32=eval_fp32)
    gs = _run(paid, torch, ctx, w.batches)
    assert ctx.last_rc == paid.OK
    g = tuple(np.concatenate([x[i] for x in gs]) for i in range(4))
    assert np.all(g[3] == 0)
    flat = W.flatten(w)
    idx = W.sample_indices(w.n, 240, seed=4321)
    o = oracle.integrate_list(flat["kind"][idx], flat["q"][idx], flat["lm"][idx],
                              flat["T"][idx], LAT, 1e-6, 1e-10, 100000, rule_n=12)
    assert_parity(tuple(x[idx] for x in g), o, 1e-6, 1e-10, flat_ident(flat, idx))
    # lower temperatures need deeper partitions
    per_T = [np.mean(x[2]) for x in gs[::2]]
    assert per_T[-1] > per_T[0]
