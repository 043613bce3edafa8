"""Training data, training, rate calibration and inference for the learned
refinement proposal (the network itself and all its arithmetic live in the
CUDA library; this module only orchestrates calls).

Targets are the rule's own relative log10 error maps of the uniform level-4
grid (paid_cell_errors); inputs are the per-integral features
(paid_mlp_features).  Training draws lattice parameters t' ~ U[-0.35, 0],
mu ~ U[-1.4, 0] and T log-uniform on [0.005, 1] (workloads.parameter_draws).
"""
from __future__ import annotations

import numpy as np

from . import paid as P
from . import workloads as W


def draw_batches(T, nq, rel_tol=1e-6, abs_tol=1e-10, max_regions=100000, device=0):
    """ph + pp batches of all 81 pairs on an nq x nq zone grid, on the device."""
    import torch
    dev = torch.device("cuda", device)
    q = torch.as_tensor(W.q_grid_bz(nq), device=dev)
    lm = torch.as_tensor(W.all_pairs(9), dtype=torch.int32, device=dev)
    return [dict(kind=k, T=float(T), q=q, lm=lm, rel_tol=rel_tol, abs_tol=abs_tol,
                 max_regions=max_regions) for k in (W.PH, W.PP)]


def features(ctx, batches):
    import torch
    return torch.cat([ctx.features(b["kind"], b["q"], b["lm"], b["T"]) for b in batches])


def targets(ctx, batches):
    import torch
    return torch.cat([ctx.cell_errors(b["kind"], b["q"], b["lm"], b["T"]) for b in batches])


def training_set(draws, nq=8, device=0):
    """(x BF16 [M, 32], target FP32 [M, 256]) over parameter draws (t', mu, T)."""
    import torch
    xs, ts = [], []
    for tp, mu, T in draws:
        ctx = P.Context(1.0, tp, mu, ffset=9, device=device)
        bs = draw_batches(T, nq, device=device)
        xs.append(features(ctx, bs))
        ts.append(targets(ctx, bs))
        ctx.close()
    return torch.cat(xs), torch.cat(ts)


def predict(prop, ctx, batches):
    """Predicted maps (FP32 [n, 256]) for batches in the global order."""
    return prop.forward(features(ctx, batches))


def calibrate_rate(prop, ctx, batches, rates=(1.5, 2.0, 3.0, 4.0, 6.0, 10.0)):
    """The seeding rate with the fewest region evaluations on these batches;
    returns (best rate, {rate: region evaluations})."""
    maps = predict(prop, ctx, batches)
    evals = {}
    for r in rates:
        ctx.integrate_multi_seeded(batches, maps, r)
        evals[r] = ctx.last_stats()["region_evals"]
    best = min(evals, key=evals.get)
    return best, evals


def train_default(device=0, n_draws=24, nq=8, epochs=30, seed=0, log=None):
    """The proposal trained on n_draws seeded parameter draws (seeds 0..n-1):
    returns (Proposal, training-loss history, seconds)."""
    import time
    import torch
    t0 = time.perf_counter()
    x, t = training_set(W.parameter_draws(n_draws, 0), nq, device)
    prop = P.Proposal(device=device, seed=seed)
    hist = prop.train(x, t, epochs=epochs, batch=4096, lr=2e-3, weight_decay=1e-4, seed=seed)
    torch.cuda.synchronize()
    if log:
        log("proposal trained on %d rows: loss %.3f -> %.3f" % (x.shape[0], hist[0], hist[-1]))
    return prop, hist, time.perf_counter() - t0


def calibrate_default(prop, device=0, n_draws=24, nq=4, t_range=(0.02, 0.3), eval_fp32=1,
                      group_mode=0):
    """Seeding rate calibrated on the training draws whose T lies in t_range
    (smaller q grid) for the given evaluation mode; returns
    (rate, {rate: summed region evaluations})."""
    tot = {}
    for tp, mu, T in W.parameter_draws(n_draws, 0):
        if not (t_range[0] <= T <= t_range[1]):
            continue
        ctx = P.Context(1.0, tp, mu, ffset=9, device=device, eval_fp32=eval_fp32,
                        group_mode=group_mode)
        _, ev = calibrate_rate(prop, ctx, draw_batches(T, nq, device=device))
        for r, e in ev.items():
            tot[r] = tot.get(r, 0) + e
        ctx.close()
    best = min(tot, key=tot.get) if tot else 4.0
    return best, tot
