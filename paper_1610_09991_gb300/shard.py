"""Splitting a list of bubble-integral batches across ranks (one GPU each).

The integrals are independent (Sec. 2 spreads them over MPI ranks by the
form-factor index for the same reason), so a multi-GPU run needs no exchange
on the data path: every rank integrates its own share and rank 0 gathers the
outputs once at the end.  The unit of the split is one q row of a batch (all
of the batch's (l, m) pairs at that q), so every share is again a list of
ordinary batches; the rows are dealt to ranks largest cost first, each to the
least-loaded rank (LPT), with ties broken by (batch, row) so that every rank
computes the same plan without talking to the others.

This module is host-side bookkeeping only: it holds none of the method's
arithmetic.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np


def row_costs(batches, cost=None):
    """Relative cost of every q row, [(batch index, row, cost)].

    `cost` may give one array per batch (one entry per q row, e.g. the region
    counts a proposal map predicts); without it a row costs npairs / sqrt(T):
    lower temperatures sharpen the Fermi surface and need deeper refinement."""
    out = []
    for b, bt in enumerate(batches):
        nq = bt.q.shape[0]
        if cost is not None:
            c = np.asarray(cost[b], dtype=np.float64).reshape(nq)
        else:
            c = np.full(nq, bt.lm.shape[0] / np.sqrt(bt.T))
        out.extend((b, r, float(c[r])) for r in range(nq))
    return out


def plan(batches, world, cost=None):
    """Rows of every batch per rank: plan[rank] = {batch index: sorted q rows}."""
    if world < 1:
        raise ValueError("world must be >= 1")
    rows = sorted(row_costs(batches, cost), key=lambda x: (-x[2], x[0], x[1]))
    load = [0.0] * world
    out = [dict() for _ in range(world)]
    for b, r, c in rows:
        k = min(range(world), key=lambda j: (load[j], j))
        load[k] += c
        out[k].setdefault(b, []).append(r)
    return [{b: np.array(sorted(v), dtype=np.int64) for b, v in sorted(p.items())} for p in out]


def local_batches(batches, share):
    """The batches of one rank's share: (batch index, sub-batch) with the
    share's q rows in ascending order and every pair of the batch."""
    return [(b, replace(batches[b], q=np.ascontiguousarray(batches[b].q[rows])))
            for b, rows in share.items()]


def assemble(batches, shares, results):
    """Full per-batch outputs from every rank's results.

    shares[k] is rank k's share and results[k] its outputs, one
    (values, errors, regions, status) tuple of numpy arrays per local batch in
    local_batches order.  Returns one such tuple per batch, in the batch's own
    order idx = iq * npairs + ip."""
    full = []
    for bt in batches:
        n = bt.n
        full.append((np.full(n, np.nan), np.full(n, np.nan), np.zeros(n, np.int64),
                     np.full(n, -1, np.int32)))
    for share, res in zip(shares, results):
        for (b, rows), r in zip(share.items(), res):
            npairs = batches[b].lm.shape[0]
            idx = (rows[:, None] * npairs + np.arange(npairs)[None, :]).reshape(-1)
            for dst, src in zip(full[b], r):
                dst[idx] = np.asarray(src).reshape(-1)
    return full


def gather(batches, shares, local_results, rank, world, group=None):
    """Collect every rank's outputs on rank 0 (torch.distributed, any backend);
    returns the assembled per-batch outputs on rank 0 and None elsewhere."""
    import torch.distributed as dist
    payload = [tuple(np.asarray(a) for a in r) for r in local_results]
    got = [None] * world if rank == 0 else None
    dist.gather_object(payload, got, dst=0, group=group)
    if rank != 0:
        return None
    return assemble(batches, shares, got)
