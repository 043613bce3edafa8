"""Training data, training, margin calibration and inference for the learned
refinement proposal (the network and all its arithmetic live in the CUDA
library; this module only orchestrates calls).

Targets are what the plain method emits: the trace of a converged unseeded
run (options.trace), per unit the level of the coarsest final region in each
of the 256 level-4 cells.  A unit is a (kind, q) group in group mode (the
headline path, one shared partition per group), else an integral.  Inputs
are the unit's features (paid_mlp_group_features / paid_mlp_features).
Training draws lattice parameters t' ~ U[-0.35, 0], mu ~ U[-1.4, 0] and T
log-uniform on [0.005, 1] (workloads.parameter_draws, seeds 0..n-1); held-out
draws use seeds 10000+.
"""
from __future__ import annotations

import numpy as np

from . import paid as P
from . import workloads as W

#: rule order and cover of the shared-partition path the proposal serves
GROUP_OPTIONS = dict(group_mode=1, rule_n=12, cover=1.0)


def _options(options):
    """Integrate options of the proposal's runs: the shared-partition path's
    rule and cover unless one partition per integral is asked for."""
    if options.get("group_mode", 1):
        return dict(GROUP_OPTIONS, **options)
    return dict(options)


def draw_batches(T, nq, rel_tol=1e-6, abs_tol=1e-10, max_regions=100000, device=0):
    """ph + pp batches of all 81 pairs on an nq x nq zone grid, on the device."""
    import torch
    dev = torch.device("cuda", device)
    q = torch.as_tensor(W.q_grid_bz(nq), device=dev)
    lm = torch.as_tensor(W.all_pairs(9), dtype=torch.int32, device=dev)
    return [dict(kind=k, T=float(T), q=q, lm=lm, rel_tol=rel_tol, abs_tol=abs_tol,
                 max_regions=max_regions) for k in (W.PH, W.PP)]


def features(ctx, batches):
    """Inputs of ctx's units for these batches (BF16 [units, 32])."""
    import torch
    if ctx.options.group_mode:
        return torch.cat([ctx.group_features(b["kind"], b["q"], b["T"]) for b in batches])
    return torch.cat([ctx.features(b["kind"], b["q"], b["lm"], b["T"]) for b in batches])


def traced_maps(ctx, batches):
    """Level maps of the final partitions of an unseeded run (FP32 [units, 256])."""
    import torch
    maps = torch.empty((ctx.units(batches), 256), dtype=torch.float32, device=ctx.torch_device)
    ctx.set_trace_buffer(maps)
    ctx.integrate_multi(batches)
    ctx.set_trace_buffer(None)
    return maps


def training_set(draws, nq=12, device=0, **options):
    """(x BF16 [M, 32], target FP32 [M, 256]) over parameter draws (t', mu, T):
    every unit of a traced plain run of each draw's ph + pp batches."""
    import torch
    xs, ts = [], []
    for tp, mu, T in draws:
        ctx = P.Context(1.0, tp, mu, ffset=9, device=device, trace=1, **options)
        bs = draw_batches(T, nq, device=device)
        xs.append(features(ctx, bs))
        ts.append(traced_maps(ctx, bs))
        ctx.close()
    return torch.cat(xs), torch.cat(ts)


def predict(prop, ctx, batches):
    """Predicted level maps (FP32 [units, 256]) for batches in the global order."""
    return prop.predict(ctx, batches)


#: temperature bands of the margin policy (upper edges) and the margins tried;
#: None = no seed (the uniform start)
T_BANDS = (0.015, 0.03, 0.045, 0.07, float("inf"))
MARGINS = (0.0, 0.5, 1.0, 2.0, None)


class MarginPolicy:
    """Seed margin per temperature band, calibrated on training draws: a
    batch at temperature T starts each cell at floor(level - margin(T)), or
    from the uniform start where the band's best choice is no seed."""

    def __init__(self, margins, bands=T_BANDS):
        self.bands = tuple(bands)
        self.margins = tuple(margins)

    def __call__(self, T):
        for edge, m in zip(self.bands, self.margins):
            if T <= edge:
                return m
        return self.margins[-1]

    def as_dict(self):
        return {("T <= %g" % e): m for e, m in zip(self.bands, self.margins)}


def seed_maps(prop, ctx, batches, policy):
    """Level maps with each batch's margin applied (for a call with margin 0):
    map - margin(T), or the context's start level everywhere (no seed)."""
    maps = predict(prop, ctx, batches)
    off = 0
    for b in batches:
        n = int(b["q"].shape[0]) * (1 if ctx.options.group_mode else int(b["lm"].shape[0]))
        m = policy(float(b["T"]))
        if m is None:
            maps[off:off + n] = float(ctx.options.init_level)
        elif m:
            maps[off:off + n] -= m
        off += n
    return maps


def integrate(prop, ctx, batches, policy, stream=None, pool_capacity=None):
    """One call under a margin policy: the seeded start when the policy gives
    a margin for some batch; the library's uniform start (streaming admission,
    no inference) when it gives None for every batch, the form the policy was
    calibrated on."""
    if all(policy(float(b["T"])) is None for b in batches):
        return ctx.integrate_multi(batches, pool_capacity=pool_capacity, stream=stream)
    return ctx.integrate_multi_seeded(batches, seed_maps(prop, ctx, batches, policy), 0.0,
                                      pool_capacity=pool_capacity, stream=stream)


def calibrate_margin(prop, ctx, batches, margins=MARGINS):
    """Region evaluations and rounds of the seeded run at each margin (None:
    the uniform start) on these batches: {margin: (region evaluations, rounds)}."""
    maps = predict(prop, ctx, batches)
    out = {}
    for mg in margins:
        if mg is None:
            ctx.integrate_multi(batches)
        else:
            ctx.integrate_multi_seeded(batches, maps, mg)
        st = ctx.last_stats()
        out[mg] = (st["region_evals"], st["rounds"])
    return out


def train_default(device=0, n_draws=192, nq=12, epochs=300, seed=0, log=None, **options):
    """The proposal trained on n_draws seeded parameter draws (seeds 0..n-1)
    for the given integrate options (default: the shared-partition path):
    returns (Proposal, training-loss history, seconds)."""
    import time
    import torch
    opts = _options(options)
    t0 = time.perf_counter()
    x, t = training_set(W.parameter_draws(n_draws, 0), nq, device, **opts)
    prop = P.Proposal(device=device, seed=seed)
    hist = prop.train(x, t, epochs=epochs, batch=1024, lr=2e-3, weight_decay=1e-4, seed=seed)
    torch.cuda.synchronize()
    if log:
        log("proposal trained on %d rows: loss %.3f -> %.3f" % (x.shape[0], hist[0], hist[-1]))
    return prop, hist, time.perf_counter() - t0


def calibrate_default(prop, device=0, n_draws=96, nq=8, **options):
    """The margin policy: per temperature band (T_BANDS) the margin of MARGINS
    with the fewest region evaluations summed over the band's training draws
    (seeds 0..n_draws-1, smaller q grid); returns (MarginPolicy, {band:
    {margin: (region evaluations, rounds)}})."""
    opts = _options(options)
    tot = [dict() for _ in T_BANDS]
    for tp, mu, T in W.parameter_draws(n_draws, 0):
        k = next(i for i, e in enumerate(T_BANDS) if T <= e)
        ctx = P.Context(1.0, tp, mu, ffset=9, device=device, **opts)
        for mg, (ev, rd) in calibrate_margin(prop, ctx, draw_batches(T, nq, device=device)).items():
            e0, r0 = tot[k].get(mg, (0, 0))
            tot[k][mg] = (e0 + ev, r0 + rd)
        ctx.close()
    best = [min(t, key=lambda m: t[m][0]) if t else None for t in tot]
    policy = MarginPolicy(best)
    return policy, {("T <= %g" % e): {str(m): v for m, v in t.items()}
                    for e, t in zip(T_BANDS, tot)}
