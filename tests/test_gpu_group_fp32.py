"""The FP32-pipe form of the shared-partition kernel (options eval_fp32 = 1
with group_mode): the kernel F, the rule's row sums and the moments in
float-float on the FP32 pipe; each region's pair values Q_2N, Q_N, their
difference, the errors and all totals in FP64.

Arithmetic level: the float-float exp and kernels against the FP64 oracle's
kernels (Sec. 2: the ph bubble F = [tanh(e1/2T) - tanh(e2/2T)] / (2 (e1 - e2))
and the Omega derivative of the flow kinds' frequency integral).  Region
level: Q_N and Q_2N of every pair against the oracle's direct nested rule
(Sec. 3).  Integral level: the usual parity criterion against the
per-integral oracle, on the full 93,312-integral flow step at the tuned rule
order and at T = 0.01 with rel tol 1e-5 and 1e-7 (the precision study).
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


def _run(torch, ctx, batches, pool_capacity=None):
    dbs = [dict(kind=b.kind, T=b.T, q=_dev(torch, b.q, torch.float64),
                lm=_dev(torch, b.lm, torch.int32), rel_tol=b.rel_tol, abs_tol=b.abs_tol,
                max_regions=b.max_regions) for b in batches]
    outs = ctx.integrate_multi(dbs, pool_capacity=pool_capacity)
    torch.cuda.synchronize()
    return [tuple(x.cpu().numpy() for x in (r.values, r.errors, r.regions, r.status)) for r in outs]


def test_float_float_exp(paid, torch):
    # relative error of e^-x against the FP64 exp: float-float carries ~2^-48,
    # the table and the polynomial ~2^-46; x itself is rounded to float-float
    # (relative 2^-49, i.e. x 2^-49 absolute in the exponent)
    ctx = paid.Context(*LAT, ffset=9)
    rng = np.random.default_rng(5)
    x = np.concatenate([np.array([0.0, 1e-30, 1e-8, 5e-3, math.log(2) / 128, 1.0, 20.0, 49.9]),
                        rng.uniform(0, 1, 20000), rng.uniform(0, 49.99, 20000),
                        np.exp(rng.uniform(-30, math.log(49.9), 20000))])
    got = ctx.check_math(2, _dev(torch, x, torch.float64)).cpu().numpy()
    ref = np.exp(-x)
    rel = np.abs(got - ref) / ref
    assert np.all(rel <= 2.0 ** -44 + x * 2.0 ** -47), (rel.max(), x[np.argmax(rel)])
    big = ctx.check_math(2, _dev(torch, np.array([50.0, 80.0, 1e9, np.nan]), torch.float64))
    big = big.cpu().numpy()
    assert np.all(big[:3] == 0.0) and np.isnan(big[3])


def _kernel_cases(rng):
    a = rng.uniform(-30, 30, 12000)
    b = rng.uniform(-30, 30, 12000)
    near_a = rng.uniform(-12, 12, 8000)
    near_b = near_a + rng.uniform(-0.07, 0.07, 8000)          # both sides of |d| = 1/16
    tiny_a = rng.uniform(-1, 1, 2000) * 1e-3
    tiny_b = -tiny_a * rng.uniform(0.5, 2, 2000)             # opposite signs near 0
    x1 = np.concatenate([a, near_a, tiny_a, [0.0, 1.0, -3.0, 0.5, 44.0, -44.0]])
    x2 = np.concatenate([b, near_b, tiny_b, [0.0, 1.0, 3.0, -0.5, 43.9, 44.0]])
    return x1, x2


def test_float_float_bubble_kernel(paid, torch):
    # 2T F(x1, x2) with x = e/2T: at T = 1/2 the oracle's F(e1, e2, T) is that
    # function of (x1, x2) = (e1, e2)
    ctx = paid.Context(*LAT, ffset=9)
    x1, x2 = _kernel_cases(np.random.default_rng(6))
    got = ctx.check_math(3, _dev(torch, x1, torch.float64), _dev(torch, x2, torch.float64))
    got = got.cpu().numpy()
    f64 = ctx.check_math(4, _dev(torch, x1, torch.float64), _dev(torch, x2, torch.float64))
    f64 = f64.cpu().numpy()
    ref = np.array([oracle.kernel_ph(a, b, 0.5) for a, b in zip(x1, x2)])
    # float-float rounding of x (2^-49 |x|) moves v = e^-|x| by 2^-49 |x| relative,
    # and the far branch's u2 - u1 (|d| > 1/16) amplifies the errors of u = v^2
    # by at most 1 / (1 - e^(-1/8)) < 8.5: |x| 2^-44 in all
    tol = (2.0 ** -43 + (np.abs(x1) + np.abs(x2)) * 2.0 ** -44) * np.abs(ref) + 1e-40
    assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) / tol)
    assert np.all(np.abs(f64 - ref) <= 1e-14 * np.abs(ref) + 1e-300)


def test_float_float_flow_kernel(paid, torch):
    ctx = paid.Context(*LAT, ffset=9)
    rng = np.random.default_rng(7)
    e1 = np.concatenate([rng.uniform(-4, 4, 10000), rng.uniform(-0.05, 0.05, 4000), [0.0, 0.2]])
    e2 = np.concatenate([rng.uniform(-4, 4, 10000), rng.uniform(-0.05, 0.05, 4000), [0.0, 0.2]])
    W = 0.1
    got = ctx.check_math(5, _dev(torch, e1, torch.float64), _dev(torch, e2, torch.float64))
    ref = np.array([oracle.kernel_flow_ph(a, b, W) for a, b in zip(e1, e2)])
    # energies of one sign: the divided difference of Hdot = 3/(4u) - 5W/(4u^2)
    # + W^2/(2u^3) (u = |e| + W) is a sum of three terms that cancel (Hdot is
    # nearly flat away from the Fermi surface), so the error scales with the
    # terms' magnitudes, not the result's; opposite signs do not cancel
    u1, u2 = np.abs(e1) + W, np.abs(e2) + W
    P, S = u1 * u2, u1 + u2
    same = (e1 < 0) == (e2 < 0)
    scale = np.where(same, 3 / (4 * P) + 5 * W * S / (4 * P * P) + W * W * (S * S + P) / (2 * P ** 3),
                     np.abs(ref))
    err = np.abs(got.cpu().numpy() - ref)
    assert np.all(err <= 2.0 ** -42 * scale + 2.0 ** -44 * np.abs(ref) + 1e-300), \
        np.max(err / (2.0 ** -42 * scale))
    f64 = ctx.check_math(6, _dev(torch, e1, torch.float64), _dev(torch, e2, torch.float64))
    assert np.all(np.abs(f64.cpu().numpy() - ref) <= 2.0 ** -48 * scale + 1e-300)


@pytest.mark.parametrize("kind,T", [(W.PH, 0.05), (W.PP, 0.01), (W.PH, 0.7), (W.OVERLAP, 1.0),
                                    (W.FLOW_PH, 0.1), (W.FLOW_PP, 0.1)])
@pytest.mark.parametrize("N", [4, 12])
def test_rule_regions_fp32_match_the_oracle_rule(paid, torch, kind, T, N):
    rng = np.random.default_rng(29 + kind + N)
    ctx = paid.Context(*LAT, ffset=9, group_mode=1, rule_n=N, eval_fp32=1)
    lm = W.all_pairs(9)
    regs = [(0, 0, 0), (1, 1, 0), (2, 3, 1)]
    for L in (3, 5, 8, 12, 20, 29):
        for _ in range(2):
            regs.append((L, int(rng.integers(0, 2 ** L)), int(rng.integers(0, 2 ** L))))
    regions = np.array(regs, dtype=np.int32)
    # the reduced energies x = e/2T are float-float (2^-49 relative): at low T
    # the row coefficient A ~ 4/2T carries an absolute error 2^-49 |A| into x
    rtol = 2e-12 * (1.0 + 0.05 / T)
    for q in (np.array([0.3, -2.1]), np.array([math.pi, 0.0])):
        q2, dq = ctx.rule_regions(kind, _dev(torch, q, torch.float64), _dev(torch, lm, torch.int32),
                                  T, _dev(torch, regions, torch.int32))
        q2, dq = q2.cpu().numpy(), dq.cpu().numpy()
        for r, (L, ix, iy) in enumerate(regs):
            ref = np.array([oracle.region_eval(kind, q, int(l), int(m), T, LAT, L, ix, iy,
                                               rule_n=N) for l, m in lm])
            # e^-|x| is flushed to zero beyond |x| = 50, so a region deep in the
            # Fermi functions' tails (all values below ~e^-50 of the kernel's
            # scale 1/4T) is held to that absolute floor, times its Jacobian
            floor = 1e-21 / T * 4.0 ** -L
            tol = rtol * (np.abs(ref).max() + 1e-300) + floor
            assert np.all(np.abs(q2[r] - ref[:, 1]) <= tol), (L, ix, iy)
            assert np.all(np.abs(dq[r] - (ref[:, 0] - ref[:, 1])) <= tol), (L, ix, iy)


def test_group_fp32_first_shell_matches_oracle(paid, torch):
    w = W.config_first_shell()
    b = w.batches[0]
    ctx = paid.Context(*w.lattice, ffset=5, group_mode=1, eval_fp32=1)
    (g,) = _run(torch, ctx, [b])
    o = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol, b.max_regions)
    assert np.all(g[3] == 0)
    assert assert_parity(g, o, b.rel_tol, b.abs_tol, batch_ident(b)) >= b.n - 1
    assert np.all(g[1] <= np.maximum(b.abs_tol, b.rel_tol * np.abs(g[0])))


@pytest.mark.parametrize("eval_fp32", [0, 1])
def test_group_full_flow_step_tuned_rule(paid, torch, eval_fp32):
    # the headline configuration at full size: all 93,312 integrals of the flow
    # step, shared partitions at N = 12, cover 1; a seeded oracle sample (same
    # rule) one by one, the pp symmetry I_lm = I_ml on every q, and (FP32
    # pipe) every integral against the FP64 group path
    w = W.config_flow_step()
    ctx = paid.Context(*w.lattice, ffset=9, group_mode=1, rule_n=12, cover=1.0,
                       eval_fp32=eval_fp32)
    gs = _run(torch, ctx, w.batches)
    g = tuple(np.concatenate([x[i] for x in gs]) for i in range(4))
    flat = W.flatten(w)
    idx = W.sample_indices(w.n, 240, seed=1234)
    o = oracle.integrate_list(flat["kind"][idx], flat["q"][idx], flat["lm"][idx],
                              flat["T"][idx], LAT, 1e-6, 1e-10, 100000, rule_n=12)
    assert_parity(tuple(x[idx] for x in g), o, 1e-6, 1e-10, flat_ident(flat, idx))
    v, e, r, s = g
    assert np.all(s == 0)
    assert np.all(e <= np.maximum(1e-10, 1e-6 * np.abs(v)))
    vpp = v[w.batches[0].n:].reshape(576, 9, 9)
    tol = 2 * np.maximum(1e-6 * np.abs(vpp), 1e-10) + 1e-12
    assert np.all(np.abs(vpp - vpp.transpose(0, 2, 1)) <= tol + tol.transpose(0, 2, 1))
    if eval_fp32:
        c64 = paid.Context(*w.lattice, ffset=9, group_mode=1, rule_n=12, cover=1.0)
        g64 = tuple(np.concatenate([x[i] for x in _run(torch, c64, w.batches)]) for i in range(4))
        c64.close()
        assert_parity(g, g64, 1e-6, 1e-10, lambda i: (int(flat["kind"][i]), flat["q"][i],
                                                      int(flat["lm"][i][0]), int(flat["lm"][i][1]),
                                                      float(flat["T"][i])))


@pytest.mark.parametrize("rel_tol", [1e-5, 1e-7])
def test_group_fp32_precision_study(paid, torch, rel_tol):
    # the flow step at T = 0.01 (the precision workload), FP32-pipe group
    # kernel at N = 12: every integral converges (none on the budget, no pool
    # exhaustion) and a seeded sample matches the oracle
    w = W.config_flow_step(T=0.01, rel_tol=rel_tol)
    ctx = paid.Context(*w.lattice, ffset=9, group_mode=1, rule_n=12, cover=1.0, eval_fp32=1)
    gs = _run(torch, ctx, w.batches)
    assert ctx.last_rc == paid.OK
    g = tuple(np.concatenate([x[i] for x in gs]) for i in range(4))
    assert np.all(g[3] == 0)
    flat = W.flatten(w)
    idx = W.sample_indices(w.n, 96, seed=1234)
    o = oracle.integrate_list(flat["kind"][idx], flat["q"][idx], flat["lm"][idx],
                              flat["T"][idx], LAT, rel_tol, 1e-10, 100000, rule_n=12)
    assert_parity(tuple(x[idx] for x in g), o, rel_tol, 1e-10, flat_ident(flat, idx))


def test_group_fp32_flow_kinds_match_oracle(paid, torch):
    w = W.config_flow_omega(nq=4)
    ctx = paid.Context(*w.lattice, ffset=9, group_mode=1, rule_n=12, cover=1.0, eval_fp32=1)
    gs = _run(torch, ctx, w.batches)
    for b, g in zip(w.batches, gs):
        assert np.all(g[3] == 0)
        idx = np.arange(0, b.n, 7)
        o = oracle.integrate_batch(b.kind, b.q, b.lm, b.T, LAT, b.rel_tol, b.abs_tol,
                                   b.max_regions, rule_n=12)
        v, e, r, s = g
        vo, eo, ro, so = o
        d = np.abs(v - vo)[idx]
        tol = np.maximum(b.rel_tol * np.abs(vo), b.abs_tol)[idx]
        # the flow kernel has a kink on the Fermi surface: disagreements beyond
        # 2 tol are decided by the h^4-Richardson trapezoid
        for i in idx[d > 2 * tol + 1e-12]:
            truth = oracle.brute_force_h4(b.kind, b.q[i // b.lm.shape[0]],
                                          int(b.lm[i % b.lm.shape[0]][0]),
                                          int(b.lm[i % b.lm.shape[0]][1]), b.T, LAT)[0]
            assert abs(v[i] - truth) <= 2 * max(b.rel_tol * abs(truth), b.abs_tol) + 1e-12


def test_group_fp32_device_loop_matches_host_loop(paid, torch):
    w = W.config_flow_step(T=0.1, nq=2)
    a = _run(torch, paid.Context(*LAT, ffset=9, group_mode=1, eval_fp32=1, device_loop=1),
             w.batches)
    b = _run(torch, paid.Context(*LAT, ffset=9, group_mode=1, eval_fp32=1, device_loop=0),
             w.batches)
    for x, y in zip(a, b):
        for u, v in zip(x, y):
            assert np.array_equal(u, v)
