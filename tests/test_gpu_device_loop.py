"""The device-resident refinement loop (one CUDA graph launch: a conditional
WHILE node around one round's kernels) against the host-driven loop.

Both run the same kernels on the same device-side loop state, and every
reduction has a fixed order, so the results must agree bit for bit: values,
errors, region counts, statuses, round counts and region-evaluation counts.
The host loop itself is held to the FP64 oracle by test_gpu_parity.py.
"""
import numpy as np
import pytest

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


def _dbs(torch, batches):
    return [dict(kind=b.kind, T=b.T,
                 q=torch.as_tensor(np.ascontiguousarray(b.q), dtype=torch.float64, device="cuda"),
                 lm=torch.as_tensor(np.ascontiguousarray(b.lm), dtype=torch.int32, device="cuda"),
                 rel_tol=b.rel_tol, abs_tol=b.abs_tol, max_regions=b.max_regions)
            for b in batches]


def _run(paid, torch, batches, seeded=False, pool_capacity=None, **opts):
    ctx = paid.Context(*LAT, ffset=9, **opts)
    dbs = _dbs(torch, batches)
    if seeded:
        outs = ctx.integrate_multi_seeded(dbs, None, 2.0, pool_capacity=pool_capacity)
    else:
        outs = ctx.integrate_multi(dbs, pool_capacity=pool_capacity)
    torch.cuda.synchronize()
    res = [tuple(x.cpu().numpy() for x in (r.values, r.errors, r.regions, r.status)) for r in outs]
    return res, ctx.last_stats(), ctx.last_rc


def _same(a, b):
    for x, y in zip(a, b):
        for u, v in zip(x, y):
            assert np.array_equal(u, v, equal_nan=True)


def _compare(paid, torch, batches, **kw):
    g, sg, rg = _run(paid, torch, batches, device_loop=1, **kw)
    h, sh, rh = _run(paid, torch, batches, device_loop=0, **kw)
    _same(g, h)
    assert rg == rh
    assert sg["graph_launches"] == 1 and sh["graph_launches"] == 0
    for k in ("rounds", "region_evals", "peak_pool", "throttled_rounds", "escalated",
              "df_regions"):
        assert sg[k] == sh[k], k
    return g, sg, rg


@pytest.mark.parametrize("fp32", [0, 1])
def test_device_loop_matches_host_loop(paid, torch, fp32):
    w = W.config_flow_step(T=0.1, nq=2)
    g, st, rc = _compare(paid, torch, w.batches, eval_fp32=fp32)
    assert rc == paid.OK
    assert st["rounds"] > 3
    assert all(np.all(np.isin(x[3], [0, 1])) for x in g)


def test_device_loop_first_shell(paid, torch):
    w = W.config_first_shell()
    g, st, rc = _compare(paid, torch, w.batches)
    assert rc == paid.OK and np.all(g[0][3] == 0)


def test_device_loop_seeded(paid, torch):
    w = W.config_flow_step(T=0.2, nq=2)
    g, st, rc = _compare(paid, torch, w.batches, seeded=True)
    assert rc == paid.OK


def test_device_loop_streaming_small_pool(paid, torch):
    # a pool far smaller than the batch's regions: admission waves and
    # throttled rounds run inside the graph exactly as in the host loop
    b = W.Batch(W.PH, 0.2, W.q_grid_bz(4), W.all_pairs(9)[::5], 1e-6, 1e-10, 100000)
    full, sf, _ = _run(paid, torch, [b])
    cap = max(sf["peak_pool"] // 3, 20000)
    g, st, rc = _compare(paid, torch, [b], pool_capacity=cap)
    assert rc == paid.OK
    assert st["peak_pool"] <= cap < sf["peak_pool"]
    assert np.array_equal(g[0][3], full[0][3])


def test_device_loop_round_cap_and_pool_full(paid, torch):
    b = W.Batch(W.PH, 0.05, W.q_grid_bz(2), W.all_pairs(5), 1e-8, 1e-12, 100000)
    g, st, rc = _compare(paid, torch, [b], max_rounds=1)
    assert rc == paid.ERR_TIMEOUT
    assert np.all(np.isin(g[0][3], [0, 3])) and np.any(g[0][3] == 3)
    g, st, rc = _compare(paid, torch, [b], pool_capacity=b.n * 16 + 64)
    assert rc == paid.ERR_POOL
    assert np.any(g[0][3] == 4)


def test_graph_is_reused_across_calls(paid, torch):
    # the second call on the same workspace layout reuses the instantiated
    # graph; its results are those of the first call
    w = W.config_flow_step(T=0.1, nq=2)
    ctx = paid.Context(*LAT, ffset=9)
    dbs = _dbs(torch, w.batches)
    a = ctx.integrate_multi(dbs)
    a = [(r.values.clone(), r.status.clone()) for r in a]
    b = ctx.integrate_multi(dbs)
    torch.cuda.synchronize()
    for (va, sa), r in zip(a, b):
        assert torch.equal(va, r.values) and torch.equal(sa, r.status)
    assert ctx.last_stats()["graph_launches"] == 1


def test_device_loop_call_is_asynchronous(paid, torch):
    # the call returns once its work is queued on the stream (the stream is
    # still busy when it returns); paid_wait gives the outcome, and the outputs
    # equal those of the synchronous form bit for bit
    w = W.config_flow_step(T=0.05, nq=12)
    dbs = _dbs(torch, w.batches)
    ctx = paid.Context(*LAT, ffset=9, group_mode=1, rule_n=12, cover=1.0, eval_fp32=1)
    sync = ctx.integrate_multi(dbs)
    ref = [r.values.clone() for r in sync]
    torch.cuda.synchronize()
    outs = ctx.integrate_multi(dbs, asynchronous=True)
    busy = not torch.cuda.current_stream().query()
    assert ctx.wait() == paid.OK
    torch.cuda.synchronize()
    assert busy
    for a, r in zip(ref, outs):
        assert torch.equal(a, r.values)
    st = ctx.last_stats()
    assert st["graph_launches"] == 1 and st["rounds"] > 2
    # a pool that cannot progress: the call itself returns OK, paid_wait
    # reports the full pool, and the unfinished integrals say so
    b = W.Batch(W.PH, 0.05, W.q_grid_bz(2), W.all_pairs(5), 1e-8, 1e-12, 100000)
    c2 = paid.Context(*LAT, ffset=9)
    (r,) = c2.integrate_multi(_dbs(torch, [b]), pool_capacity=b.n * 16 + 64, asynchronous=True)
    assert c2.wait() == paid.ERR_POOL
    assert (r.status == 4).any()
