"""Truncated-unity products (Eqs. matmul-P/C/D) on the GPU against the oracle,
including the flow-step use: the bubble matrices straight from an integrate
call (pairs all (l, m), l-major) as X."""
import numpy as np
import pytest

import oracle
from paper_1610_09991_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("nff", [1, 5, 9])
def test_tu_products_match_oracle(paid, torch, nff):
    rng = np.random.default_rng(nff)
    nq = 777
    m = [rng.normal(size=(nq, nff, nff)) for _ in range(5)]
    ctx = paid.Context(*W.LATTICE, ffset=9)
    got = ctx.tu_flow_rhs(*[torch.as_tensor(a, device="cuda") for a in m])
    want = oracle.tu_flow_rhs(*m)
    for g, w_ in zip(got, want):
        assert np.allclose(g.cpu().numpy(), w_, rtol=1e-13, atol=1e-13)


def test_tu_products_on_integrated_bubbles(paid, torch):
    w = W.config_flow_step(T=0.2, nq=3)
    ctx = paid.Context(*w.lattice, ffset=9, group_mode=1, rule_n=12, cover=1.0)
    dbs = [dict(kind=b.kind, T=b.T, q=torch.as_tensor(b.q, device="cuda"),
                lm=torch.as_tensor(b.lm, dtype=torch.int32, device="cuda"),
                rel_tol=b.rel_tol, abs_tol=b.abs_tol, max_regions=b.max_regions)
           for b in w.batches]
    ph, pp = ctx.integrate_multi(dbs)
    nq = w.batches[0].q.shape[0]
    Xph = ph.values.view(nq, 9, 9)
    Xpp = pp.values.view(nq, 9, 9)
    rng = np.random.default_rng(1)
    V = [torch.as_tensor(rng.normal(size=(nq, 9, 9)), device="cuda") for _ in range(3)]
    got = ctx.tu_flow_rhs(V[0], V[1], V[2], Xpp.contiguous(), Xph.contiguous())
    want = oracle.tu_flow_rhs(*[v.cpu().numpy() for v in V], Xpp.cpu().numpy(), Xph.cpu().numpy())
    for g, w_ in zip(got, want):
        assert np.allclose(g.cpu().numpy(), w_, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("group_mode", [1, 2])
def test_tu_products_fused_into_the_flow_step(paid, torch, group_mode):
    # the truncated-unity right-hand sides formed inside the integrate call as
    # each (kind, l) group finishes, against the oracle's products of the
    # bubbles that same call returns; the call launches no separate product
    # kernel
    w = W.config_flow_omega(omega=0.2, nq=3)
    ctx = paid.Context(*w.lattice, ffset=9, group_mode=group_mode, rule_n=12, cover=1.0,
                       eval_fp32=1)
    nq = w.batches[0].q.shape[0]
    rng = np.random.default_rng(7)
    V = [torch.as_tensor(rng.normal(size=(nq, 9, 9)), device="cuda") for _ in range(3)]
    out = [torch.full((nq, 9, 9), float("nan"), dtype=torch.float64, device="cuda")
           for _ in range(3)]
    dbs = []
    for b in w.batches:
        d = dict(kind=b.kind, T=b.T, q=torch.as_tensor(b.q, device="cuda"),
                 lm=torch.as_tensor(b.lm, dtype=torch.int32, device="cuda"),
                 rel_tol=b.rel_tol, abs_tol=b.abs_tol, max_regions=b.max_regions)
        if b.kind == W.FLOW_PP:
            d.update(tu_v=(V[0],), tu_out=(out[0],))
        else:
            d.update(tu_v=(V[1], V[2]), tu_out=(out[1], out[2]))
        dbs.append(d)
    res = ctx.integrate_multi(dbs)
    torch.cuda.synchronize()
    st = ctx.last_stats()
    Xph = res[[b.kind for b in w.batches].index(W.FLOW_PH)].values.view(nq, 9, 9).cpu().numpy()
    Xpp = res[[b.kind for b in w.batches].index(W.FLOW_PP)].values.view(nq, 9, 9).cpu().numpy()
    want = oracle.tu_flow_rhs(*[v.cpu().numpy() for v in V], Xpp, Xph)
    for g, w_ in zip(out, want):
        assert np.allclose(g.cpu().numpy(), w_, rtol=1e-12, atol=1e-13)
    # the products came with the loop: the call's kernels are the loop's
    plain = paid.Context(*w.lattice, ffset=9, group_mode=group_mode, rule_n=12, cover=1.0,
                         eval_fp32=1)
    plain.integrate_multi([{k: v for k, v in d.items() if k not in ("tu_v", "tu_out")}
                           for d in dbs])
    assert st["launches"] == plain.last_stats()["launches"]
    # pairs out of l-major order: NaN products, not wrong ones
    perm = dbs[0]["lm"].flip(0).contiguous()
    bad = [dict(dbs[0], lm=perm)]
    for t in bad[0]["tu_out"]:
        t.zero_()
    ctx.integrate_multi(bad)
    torch.cuda.synchronize()
    assert all(torch.isnan(t).all() for t in bad[0]["tu_out"])
