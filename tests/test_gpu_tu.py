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
