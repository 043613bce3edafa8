"""The allocation-free entry point, paid_integrate_batch_static.

It serves callers that cannot allocate device memory when they integrate
(a runtime with a device-memory budget fixed at start-up, a plug-in inside
another framework's memory manager, a loop that must not allocate): the region
pool is a fixed 64 MiB array inside the library instead of a caller workspace.
This file checks, through the C ABI, that two calls in a row give the same
results as paid_integrate_batch (the second call runs on the scratch the first
one left behind), and that a batch beyond the stated maximum, or one that
breaks paid_integrate_batch's own argument rules, is refused.  It is named to
be collected last, and passes both alone in a fresh process and after the rest
of the suite.
"""
import ctypes

import numpy as np
import pytest

from paper_1610_09991_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_09991_gb300 import build as B
    B.build()
    from paper_1610_09991_gb300 import paid as P
    return torch, P


def _within(a, b, rel, ab):
    return np.all(np.abs(a - b) <= 2 * np.maximum(rel * np.abs(b), ab) + 1e-12)


def test_static_matches_workspace_entry_twice(env):
    torch, P = env
    w = W.config_first_shell()          # 400 ph integrals at T = 0.5
    b = w.batches[0]
    ctx = P.Context(*w.lattice, ffset=5)
    q = torch.as_tensor(b.q, device="cuda")
    lm = torch.as_tensor(b.lm, dtype=torch.int32, device="cuda")
    ref = ctx.integrate_batch(b.kind, q, lm, b.T, b.rel_tol, b.abs_tol, b.max_regions)
    torch.cuda.synchronize()
    rv, rs = ref.values.cpu().numpy(), ref.status.cpu().numpy()
    for _ in range(2):
        out = ctx.integrate_batch_static(b.kind, q, lm, b.T, b.rel_tol, b.abs_tol, b.max_regions)
        torch.cuda.synchronize()
        assert ctx.last_rc == P.OK
        v, s = out.values.cpu().numpy(), out.status.cpu().numpy()
        assert np.array_equal(s, rs)
        assert _within(v, rv, b.rel_tol, b.abs_tol)
        assert np.array_equal(out.regions.cpu().numpy(), ref.regions.cpu().numpy())


def test_static_rejects_batches_beyond_its_maximum(env):
    torch, P = env
    ctx = P.Context(*W.LATTICE, ffset=9)
    q = torch.zeros((64, 2), dtype=torch.float64, device="cuda")
    lm = torch.as_tensor(W.all_pairs(9), dtype=torch.int32, device="cuda")   # 64 * 81 > 4096
    with pytest.raises(P.PaidError) as ei:
        ctx.integrate_batch_static(P.PH, q, lm, 0.5)
    assert ei.value.rc == P.ERR_ARG


def test_static_applies_the_same_argument_rules(env):
    torch, P = env
    ctx = P.Context(*W.LATTICE, ffset=9, group_mode=1)
    q = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    lm = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    for omega in (0.0, -0.1, float("nan")):        # the flow kinds need Omega > 0
        with pytest.raises(P.PaidError) as ei:
            ctx.integrate_batch_static(P.FLOW_PH, q, lm, omega)
        assert ei.value.rc == P.ERR_ARG
    with pytest.raises(ValueError):                # the binding checks layouts first
        ctx.integrate_batch_static(P.PH, q.float(), lm, 0.5)
    with pytest.raises(ValueError):
        ctx.integrate_batch_static(P.PH, q, lm.long(), 0.5)
