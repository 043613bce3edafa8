"""The Omega-regulated flow kinds (Sec. 2 regulator; the frequency integrals
of Eqs. chi_ph / chi_pp done analytically, differentiated in Omega) in the
shared-partition kernel, against the FP64 oracle: region by region (the rule
on given regions, every pair), integral by integral (2 tol criterion), and
through the truncated-unity products of one flow step."""
import math

import numpy as np
import pytest

import oracle
from paper_1610_09991_gb300 import workloads as W
from tests.test_gpu_parity import assert_parity, batch_ident

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


@pytest.mark.parametrize("kind", [W.FLOW_PH, W.FLOW_PP])
@pytest.mark.parametrize("om", [0.05, 0.5])
def test_flow_rule_regions_match_oracle(paid, torch, kind, om):
    rng = np.random.default_rng(kind * 7 + int(om * 100))
    lm = W.all_pairs(9)
    regs = [(0, 0, 0), (2, 1, 3)] + [(L, int(rng.integers(0, 2 ** L)), int(rng.integers(0, 2 ** L)))
                                     for L in (4, 7, 11, 16) for _ in range(2)]
    for N in (4, 12):
        ctx = paid.Context(*LAT, ffset=9, group_mode=1, rule_n=N)
        for q in (np.array([0.6, -1.7]), np.array([math.pi, math.pi])):
            q2, dq = ctx.rule_regions(kind, _dev(torch, q, torch.float64),
                                      _dev(torch, lm, torch.int32), om,
                                      _dev(torch, np.array(regs, dtype=np.int32), torch.int32))
            q2, dq = q2.cpu().numpy(), dq.cpu().numpy()
            for r, (L, ix, iy) in enumerate(regs):
                ref = np.array([oracle.region_eval(kind, q, int(l), int(m), om, LAT, L, ix, iy,
                                                   rule_n=N) for l, m in lm])
                scale = np.abs(ref).max() + 1e-300
                assert np.all(np.abs(q2[r] - ref[:, 1]) <= 1e-12 * scale), (N, L, ix, iy)
                assert np.all(np.abs(dq[r] - (ref[:, 0] - ref[:, 1])) <= 1e-12 * scale)


@pytest.mark.parametrize("om", [0.05, 0.3])
def test_flow_integrals_match_oracle(paid, torch, om):
    w = W.config_flow_omega(omega=om, nq=4)
    ctx = paid.Context(*w.lattice, ffset=9, group_mode=1, rule_n=12, cover=1.0)
    dbs = [dict(kind=b.kind, T=b.T, q=_dev(torch, b.q, torch.float64),
                lm=_dev(torch, b.lm, torch.int32), rel_tol=b.rel_tol, abs_tol=b.abs_tol,
                max_regions=b.max_regions) for b in w.batches]
    outs = ctx.integrate_multi(dbs)
    torch.cuda.synchronize()
    assert ctx.last_rc == paid.OK
    for b, r in zip(w.batches, outs):
        g = tuple(x.cpu().numpy() for x in (r.values, r.errors, r.regions, r.status))
        assert np.all(np.isin(g[3], [0, 1]))
        # the oracle with the same rule: at N = 4 the pairs that vanish by
        # symmetry exhaust its region budget at small Omega
        o = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol,
                                   b.max_regions, rule_n=12)
        assert assert_parity(g, o, b.rel_tol, b.abs_tol, batch_ident(b)) >= 0.9 * b.n
        # f_l(k) f_m(k): the bubble matrices are symmetric
        v = g[0].reshape(-1, 9, 9)
        tol = 2 * np.maximum(1e-6 * np.abs(v), 1e-10) + 1e-12
        assert np.all(np.abs(v - v.transpose(0, 2, 1)) <= tol + tol.transpose(0, 2, 1))


def test_flow_kinds_need_group_mode(paid, torch):
    ctx = paid.Context(*LAT, ffset=9)
    dbs = [dict(kind=W.FLOW_PH, T=0.1, q=_dev(torch, np.zeros((1, 2)), torch.float64),
                lm=_dev(torch, np.array([(0, 0)]), torch.int32))]
    with pytest.raises(paid.PaidError):
        ctx.integrate_multi(dbs)


def test_one_flow_step_rhs(paid, torch):
    # dP, dC, dD of Eqs. matmul-P/C/D from the GPU bubbles, against the oracle's
    # products of the oracle's bubbles (both at tolerance: compared at 4 tol)
    w = W.config_flow_omega(omega=0.2, nq=2)
    ctx = paid.Context(*w.lattice, ffset=9, group_mode=1, rule_n=12, cover=1.0)
    dbs = [dict(kind=b.kind, T=b.T, q=_dev(torch, b.q, torch.float64),
                lm=_dev(torch, b.lm, torch.int32), rel_tol=1e-9, abs_tol=1e-12,
                max_regions=b.max_regions) for b in w.batches]
    ph, pp = ctx.integrate_multi(dbs)
    nq = w.batches[0].q.shape[0]
    rng = np.random.default_rng(4)
    V = [rng.normal(size=(nq, 9, 9)) for _ in range(3)]
    got = ctx.tu_flow_rhs(*[_dev(torch, v, torch.float64) for v in V],
                          pp.values.view(nq, 9, 9).contiguous(), ph.values.view(nq, 9, 9).contiguous())
    bo = [oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, 1e-9, 1e-12, b.max_regions,
                                 rule_n=12)[0] for b in w.batches]
    want = oracle.tu_flow_rhs(*V, bo[1].reshape(nq, 9, 9), bo[0].reshape(nq, 9, 9))
    for g, w_ in zip(got, want):
        g = g.cpu().numpy()
        scale = np.abs(w_).max()
        assert np.all(np.abs(g - w_) <= 1e-7 * scale)
