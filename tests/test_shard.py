"""The multi-rank path on CPU: the shard plan, and two gloo ranks that each
integrate their share with the FP64 oracle and gather on rank 0, against one
process integrating everything.  The oracle is deterministic per integral, so
the gathered outputs must equal the single-process ones exactly."""
import os
import socket

import numpy as np
import pytest

from paper_1610_09991_gb300 import shard as S
from paper_1610_09991_gb300 import workloads as W


def _batches():
    w = W.config_flow_step(T=0.5, nq=3)          # 2 x 9 q x 81 pairs
    fs = W.config_first_shell().batches[0]
    return w.batches + [W.Batch(fs.kind, fs.T, fs.q, fs.lm, fs.rel_tol, fs.abs_tol, fs.max_regions)]


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_plan_is_a_balanced_partition(world):
    bs = _batches()
    p = S.plan(bs, world)
    seen = {}
    for share in p:
        for b, rows in share.items():
            assert np.all(np.diff(rows) > 0)
            for r in rows:
                assert (b, int(r)) not in seen
                seen[(b, int(r))] = True
    assert len(seen) == sum(b.q.shape[0] for b in bs)
    costs = S.row_costs(bs)
    cmap = {(b, r): c for b, r, c in costs}
    loads = [sum(cmap[(b, int(r))] for b, rows in share.items() for r in rows) for share in p]
    assert max(loads) - min(loads) <= max(c for _, _, c in costs) + 1e-9
    # the same plan on every rank
    assert all(all(np.array_equal(x[b], y[b]) for b in x) and x.keys() == y.keys()
               for x, y in zip(p, S.plan(bs, world)))


def test_assemble_restores_the_global_order():
    bs = _batches()
    p = S.plan(bs, 3)
    results = []
    for share in p:
        res = []
        for b, sub in S.local_batches(bs, share):
            rows = share[b]
            npairs = sub.lm.shape[0]
            gidx = (rows[:, None] * npairs + np.arange(npairs)[None, :]).reshape(-1)
            res.append((gidx + 1000.0 * b, -gidx.astype(float), gidx, np.zeros_like(gidx, np.int32)))
        results.append(res)
    full = S.assemble(bs, p, results)
    for b, bt in enumerate(bs):
        assert np.array_equal(full[b][0], np.arange(bt.n) + 1000.0 * b)
        assert np.array_equal(full[b][2], np.arange(bt.n))
        assert np.all(full[b][3] == 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out, group_global=False):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bs = _batches()
        shares = S.plan(bs, world)
        local = []
        run = oracle.integrate_group_global if group_global else oracle.integrate_batch
        for b, sub in S.local_batches(bs, shares[rank]):
            local.append(run(sub.kind, sub.q, sub.lm, sub.T, W.LATTICE, sub.rel_tol,
                             sub.abs_tol, sub.max_regions, nthreads=1))
        full = S.gather(bs, shares, local, rank, world)
        if rank == 0:
            np.savez(out, *[a for r in full for a in r])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("group_global", [False, True])
def test_two_gloo_ranks_match_one_process(tmp_path, group_global):
    # per-integral Algorithm 1, and Algorithm 2's group error: a shard is a set
    # of q rows, each row is a whole (kind, q) group, so no group sum crosses
    # ranks and the gathered results equal one process's bit for bit
    import torch.multiprocessing as mp
    import oracle
    out = str(tmp_path / "gathered.npz")
    mp.start_processes(_rank, args=(2, _free_port(), out, group_global), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(out)
    arrays = [got["arr_%d" % i] for i in range(len(got.files))]
    bs = _batches()
    run = oracle.integrate_group_global if group_global else oracle.integrate_batch
    for b, bt in enumerate(bs):
        ref = run(bt.kind, bt.q, bt.lm, bt.T, W.LATTICE, bt.rel_tol, bt.abs_tol, bt.max_regions)
        for j in range(4):
            assert np.array_equal(arrays[4 * b + j], ref[j]), (b, j)
