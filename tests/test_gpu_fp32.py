"""GPU parity of the FP32-evaluation path (integrand in FP32, energies, rule
sums, error differences and totals in FP64, per-region rounding-noise bound,
FP64 re-evaluation of integrals whose noise exceeds half their tolerance).

Same criterion as the FP64 path: integrals both sides report CONVERGED agree
within 2 max(rel_tol |v|, abs_tol) + 1e-12 of the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1610_09991_gb300 import workloads as W
from tests.test_gpu_parity import assert_parity, batch_ident, flat_ident, run_gpu

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


def test_fp32_first_shell_matches_oracle(paid, torch):
    w = W.config_first_shell()
    b = w.batches[0]
    ctx = paid.Context(*w.lattice, ffset=5, eval_fp32=1)
    (g,) = run_gpu(paid, torch, ctx, [b])
    o = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol, b.max_regions)
    assert np.all(g[3] == 0)
    assert assert_parity(g, o, b.rel_tol, b.abs_tol, batch_ident(b)) >= b.n - 1


def test_fp32_flow_step_small_grid_matches_oracle(paid, torch):
    w = W.config_flow_step(T=0.05, nq=4)
    ctx = paid.Context(*w.lattice, ffset=9, eval_fp32=1)
    gs = run_gpu(paid, torch, ctx, w.batches)
    for b, g in zip(w.batches, gs):
        o = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol,
                                   b.max_regions)
        assert assert_parity(g, o, b.rel_tol, b.abs_tol, batch_ident(b)) >= 0.9 * b.n


def test_fp32_full_flow_step_against_fp64_gpu_and_oracle(paid, torch):
    w = W.config_flow_step()
    c64 = paid.Context(*w.lattice, ffset=9)
    c32 = paid.Context(*w.lattice, ffset=9, eval_fp32=1)
    g64 = run_gpu(paid, torch, c64, w.batches)
    g32 = run_gpu(paid, torch, c32, w.batches)
    cat = lambda gs: tuple(np.concatenate([x[i] for x in gs]) for i in range(4))
    a64, a32 = cat(g64), cat(g32)
    flat = W.flatten(w)
    every = np.arange(w.n)
    # every integral: both converged results lie within 2 tol of each other
    # (a disagreement is decided by brute force, which the FP32 side must match)
    assert_parity(a32, a64, 1e-6, 1e-10, flat_ident(flat, every), max_adjudicated=1e-4)
    idx = W.sample_indices(w.n, 240, seed=4321)
    o = oracle.integrate_list(flat["kind"][idx], flat["q"][idx], flat["lm"][idx],
                              flat["T"][idx], LAT, 1e-6, 1e-10, 100000)
    assert_parity(tuple(x[idx] for x in a32), o, 1e-6, 1e-10, flat_ident(flat, idx))
    # the FP32 path does not need more regions than the FP64 path
    assert a32[2].sum() <= 1.1 * a64[2].sum()


@pytest.mark.parametrize("rel_tol", [1e-5, 1e-7])
def test_fp32_low_T_sample(paid, torch, rel_tol):
    # the flow-step batch at T = 0.01, on a seeded sample of 96 integrals
    w = W.config_flow_step(T=0.01, rel_tol=rel_tol)
    flat = W.flatten(w)
    idx = W.sample_indices(w.n, 96, seed=1234)
    qs = flat["q"][idx]
    lms = flat["lm"][idx]
    kinds = flat["kind"][idx]
    ctx = paid.Context(*w.lattice, ffset=9, eval_fp32=1)
    bs = [W.Batch(int(k), 0.01, qs[i:i + 1], lms[i:i + 1], rel_tol, 1e-10, 100000)
          for i, k in enumerate(kinds)]
    gs = run_gpu(paid, torch, ctx, bs)
    g = tuple(np.concatenate([x[i] for x in gs]) for i in range(4))
    o = oracle.integrate_list(kinds, qs, lms, 0.01, LAT, rel_tol, 1e-10, 100000)
    assert_parity(g, o, rel_tol, 1e-10, flat_ident(flat, idx))


def test_fp32_escalates_to_fp64_when_noise_exceeds_tolerance(paid, torch):
    # tolerances far below FP32 resolution: every integral must be finished in FP64
    b = W.Batch(W.PH, 0.3, W.q_grid_bz(2), W.all_pairs(5)[::2], 1e-11, 1e-15, 100000)
    c32 = paid.Context(*LAT, ffset=5, eval_fp32=1)
    c64 = paid.Context(*LAT, ffset=5)
    (g32,) = run_gpu(paid, torch, c32, [b])
    (g64,) = run_gpu(paid, torch, c64, [b])
    o = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol, b.max_regions)
    assert assert_parity(g32, o, b.rel_tol, b.abs_tol, batch_ident(b)) > 0
    assert assert_parity(g32, g64, b.rel_tol, b.abs_tol, batch_ident(b)) > 0
    assert c32.last_stats()["escalated"] > 0
