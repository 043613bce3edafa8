"""GPU tests of the learned refinement proposal: the BF16 tensor-core network
against the FP64 reference (oracle/mlp.py), the training targets against the
oracle's region rule, seeding that never changes what the cubature returns,
and the gain of a trained network over the unseeded start."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_1610_09991_gb300 import workloads as W
from tests.test_gpu_parity import assert_parity, batch_ident, run_gpu

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


def _bf16_round(a):
    import torch
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def test_forward_and_gradient_match_fp64_reference(paid, torch):
    prop = paid.Proposal(seed=3)
    rng = np.random.default_rng(0)
    M = 300
    x = torch.as_tensor(rng.normal(size=(M, 32)), dtype=torch.bfloat16, device="cuda")
    t = torch.as_tensor(rng.normal(size=(M, 256)), dtype=torch.float32, device="cuda")
    y = prop.forward(x)
    g, loss = prop.grad(x, t)
    torch.cuda.synchronize()
    p64 = prop.state().astype(np.float64)
    # the reference sees the BF16-rounded weights and inputs the kernels use
    pr = p64.copy()
    o = 0
    for k, n in omlp.layer_shapes():
        pr[o:o + k * n] = _bf16_round(p64[o:o + k * n])
        o += k * n + n
    xr = x.float().double().cpu().numpy()
    yr, _ = omlp.forward(pr, xr)
    yg = y.double().cpu().numpy()
    scale = np.abs(yr).mean()
    assert np.abs(yg - yr).max() <= 0.05 * scale + 0.02 * np.abs(yr).max()
    lr, gr = omlp.loss_and_grad(pr, xr, t.double().cpu().numpy())
    gg = g.double().cpu().numpy()
    assert abs(float(loss.item()) - lr) <= 0.02 * lr
    rel = np.linalg.norm(gg - gr) / np.linalg.norm(gr)
    cos = float(gg @ gr / (np.linalg.norm(gg) * np.linalg.norm(gr)))
    assert rel < 0.05 and cos > 0.998, (rel, cos)


def test_training_reduces_loss(paid, torch):
    prop = paid.Proposal(seed=1)
    rng = np.random.default_rng(2)
    M = 8192
    xn = rng.normal(size=(M, 32))
    tn = np.tanh(xn[:, :8] @ rng.normal(size=(8, 256)) / 3.0)
    x = torch.as_tensor(xn, dtype=torch.bfloat16, device="cuda")
    t = torch.as_tensor(tn, dtype=torch.float32, device="cuda")
    hist = prop.train(x, t, epochs=8, batch=1024, lr=2e-3)
    assert hist[-1] < 0.3 * hist[0]


def test_cell_error_targets_match_oracle_rule(paid, torch):
    ctx = paid.Context(*LAT, ffset=9)
    q = np.array([(0.4, -1.3)])
    lm = np.array([(1, 3), (0, 0)], dtype=np.int32)
    for kind in (W.PH, W.PP):
        m = ctx.cell_errors(kind, torch.as_tensor(q, device="cuda"),
                            torch.as_tensor(lm, dtype=torch.int32, device="cuda"), 0.1)
        torch.cuda.synchronize()
        m = m.cpu().numpy()
        for ip, (l, mm) in enumerate(lm):
            qs = [oracle.region_eval(kind, q[0], l, mm, 0.1, LAT, 4, ix, iy)
                  for ix in range(16) for iy in range(16)]
            err = np.array([abs(a - b) for a, b in qs])
            S = sum(abs(b) for a, b in qs)
            want = np.clip(np.log10(np.maximum(err / S, 1e-16)), -16, 0)
            got = m[ip]
            big = want > -12
            assert np.abs(got[big] - want[big]).max() < 1e-3


@pytest.mark.parametrize("mode", ["uniform4", "exact", "random"])
def test_seeded_start_keeps_parity(paid, torch, mode):
    b = W.Batch(W.PH, 0.05, W.q_grid_bz(2), W.all_pairs(9)[::4], 1e-6, 1e-10, 100000)
    ctx = paid.Context(*LAT, ffset=9, eval_fp32=1)
    q = torch.as_tensor(b.q, device="cuda")
    lm = torch.as_tensor(b.lm, dtype=torch.int32, device="cuda")
    if mode == "uniform4":
        prop = None
    elif mode == "exact":
        prop = ctx.cell_errors(b.kind, q, lm, b.T)
    else:
        g = torch.Generator(device="cpu").manual_seed(5)
        prop = (torch.rand((b.n, 256), generator=g) * -16.0).to("cuda")
    (r,) = ctx.integrate_multi_seeded([dict(kind=b.kind, T=b.T, q=q, lm=lm, rel_tol=b.rel_tol,
                                            abs_tol=b.abs_tol, max_regions=b.max_regions)],
                                      prop, 2.0)
    torch.cuda.synchronize()
    g = tuple(x.cpu().numpy() for x in (r.values, r.errors, r.regions, r.status))
    o = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol, b.max_regions)
    # whatever the map, every converged result is right; a useless map may
    # only cost regions (integrals that run into the budget stay within
    # E_gpu + E_oracle of the oracle)
    n = assert_parity(g, o, b.rel_tol, b.abs_tol, batch_ident(b))
    if mode != "random":
        assert n >= 0.9 * b.n


def test_trained_proposal_gains_over_unseeded_start(paid, torch):
    from paper_1610_09991_gb300 import proposal as PR
    prop, hist, secs = PR.train_default(n_draws=8, nq=6, epochs=20)
    assert hist[-1] < hist[0]
    tp, mu, T = W.parameter_draws(1, 10000)[0]
    ctx = paid.Context(1.0, tp, mu, ffset=9, eval_fp32=1)
    bs = PR.draw_batches(T, 8)
    rate, evals = PR.calibrate_rate(prop, ctx, bs)
    plain = ctx.integrate_multi(bs)
    st_plain = ctx.last_stats()
    maps = PR.predict(prop, ctx, bs)
    seeded = ctx.integrate_multi_seeded(bs, maps, rate)
    st_seed = ctx.last_stats()
    uni = ctx.integrate_multi_seeded(bs, None, rate)
    st_uni = ctx.last_stats()
    torch.cuda.synchronize()
    # same accuracy: both within 2 tol of each other on every converged integral
    for a, c in zip(seeded, plain):
        ga = tuple(x.cpu().numpy() for x in (a.values, a.errors, a.regions, a.status))
        gc = tuple(x.cpu().numpy() for x in (c.values, c.errors, c.regions, c.status))
        both = (ga[3] == 0) & (gc[3] == 0)
        tol = np.maximum(1e-6 * np.abs(gc[0]), 1e-10)
        assert np.mean(np.abs(ga[0] - gc[0])[both] <= 2 * tol[both] + 1e-12) > 0.999
    print("rate", rate, evals, "rounds plain/seeded/uniform4", st_plain["rounds"], st_seed["rounds"],
          st_uni["rounds"], "region evals", st_plain["region_evals"], st_seed["region_evals"],
          st_uni["region_evals"])
    # the calibrated trained seed skips early rounds at a bounded cost in
    # regions (a per-cell depth cannot follow a line-shaped Fermi surface, so
    # calibration keeps the seed shallow)
    assert st_seed["rounds"] < st_plain["rounds"]
    assert st_seed["region_evals"] <= 1.10 * st_plain["region_evals"]


@pytest.mark.parametrize("mode", ["uniform4", "exact", "random"])
def test_group_seeded_start_keeps_parity(paid, torch, mode):
    # shared-partition mode: a group is seeded from the cell-wise largest value
    # of its pairs' maps; the result must not depend on the map's quality
    b = W.Batch(W.PP, 0.05, W.q_grid_bz(2), W.all_pairs(9), 1e-6, 1e-10, 100000)
    ctx = paid.Context(*LAT, ffset=9, group_mode=1)
    q = torch.as_tensor(b.q, device="cuda")
    lm = torch.as_tensor(b.lm, dtype=torch.int32, device="cuda")
    if mode == "uniform4":
        prop = None
    elif mode == "exact":
        prop = ctx.cell_errors(b.kind, q, lm, b.T)
    else:
        g = torch.Generator(device="cpu").manual_seed(5)
        prop = (torch.rand((b.n, 256), generator=g) * -16.0).to("cuda")
    (r,) = ctx.integrate_multi_seeded([dict(kind=b.kind, T=b.T, q=q, lm=lm, rel_tol=b.rel_tol,
                                            abs_tol=b.abs_tol, max_regions=b.max_regions)],
                                      prop, 2.0)
    torch.cuda.synchronize()
    g = tuple(x.cpu().numpy() for x in (r.values, r.errors, r.regions, r.status))
    o = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol, b.max_regions)
    n = assert_parity(g, o, b.rel_tol, b.abs_tol, batch_ident(b))
    if mode != "random":
        assert n >= 0.9 * b.n


def test_trained_proposal_in_group_mode(paid, torch):
    from paper_1610_09991_gb300 import proposal as PR
    prop, hist, secs = PR.train_default(n_draws=8, nq=6, epochs=20)
    tp, mu, T = W.parameter_draws(1, 10000)[0]
    ctx = paid.Context(1.0, tp, mu, ffset=9, group_mode=1)
    bs = PR.draw_batches(T, 8)
    rate, evals = PR.calibrate_rate(prop, ctx, bs)
    plain = ctx.integrate_multi(bs)
    st_plain = ctx.last_stats()
    maps = PR.predict(prop, ctx, bs)
    seeded = ctx.integrate_multi_seeded(bs, maps, rate)
    st_seed = ctx.last_stats()
    torch.cuda.synchronize()
    for a, c in zip(seeded, plain):
        va, sa = a.values.cpu().numpy(), a.status.cpu().numpy()
        vc, sc = c.values.cpu().numpy(), c.status.cpu().numpy()
        both = (sa == 0) & (sc == 0)
        tol = np.maximum(1e-6 * np.abs(vc), 1e-10)
        assert np.mean(np.abs(va - vc)[both] <= 2 * tol[both] + 1e-12) > 0.999
    print("group rate", rate, evals, "rounds plain/seeded", st_plain["rounds"], st_seed["rounds"],
          "region evals", st_plain["region_evals"], st_seed["region_evals"])
    # in group mode the seed skips early rounds but costs regions: a group is
    # seeded as deep as its most demanding pair asks, cell by cell, while the
    # unseeded group refines from the 16-region start only where the shared
    # selection needs it (measured: 8 -> 6 rounds for ~19 % more region
    # evaluations at the calibrated rate); the bound guards that trade
    assert st_seed["rounds"] < st_plain["rounds"]
    assert st_seed["region_evals"] <= 1.30 * st_plain["region_evals"]
