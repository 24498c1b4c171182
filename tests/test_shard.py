"""Sharding of a batch of independent systems across ranks (CPU, gloo, world size 2).

Every rank computes the partition on its own and builds only its systems; the ranks
exchange nothing but what the test gathers to check: together they hold every system of
the batch exactly once, with the particles of the full batch, at balanced cost."""
import os
import socket

import numpy as np
import pytest

from paper_2107_07166_gb300 import shard, synth


def test_lpt_partition_is_a_balanced_partition():
    sizes, _ = synth.batch_sizes(1024, 1000)
    for n_parts in (1, 2, 3, 8):
        parts = shard.lpt_partition(sizes, n_parts)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(len(sizes)))
        cost = [shard.system_cost(sizes[p]).sum() for p in parts]
        # greedy LPT stays within the largest single system of the mean load
        assert max(cost) - min(cost) <= shard.system_cost(sizes).max()
        # deterministic: the same sizes give the same groups
        again = shard.lpt_partition(sizes, n_parts)
        assert all(np.array_equal(a, b) for a, b in zip(parts, again))
    with pytest.raises(ValueError):
        shard.lpt_partition(sizes, 0)


def test_batch_subset_matches_full_batch():
    x, m, off = synth.batch(9, 400, 100, 3000)
    idx = np.array([0, 3, 4, 8])
    xs, ms, offs = synth.batch_subset(9, 400, idx, 100, 3000)
    for k, i in enumerate(idx):
        assert np.array_equal(xs[offs[k]:offs[k + 1]], x[off[i]:off[i + 1]])
        assert np.array_equal(ms[offs[k]:offs[k + 1]], m[off[i]:off[i + 1]])
    xe, me, oe = synth.batch_subset(9, 400, np.array([], dtype=np.int64), 100, 3000)
    assert xe.shape == (0, 3) and me.shape == (0,) and np.array_equal(oe, [0])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_sys, seed, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes, _ = synth.batch_sizes(n_sys, seed, 100, 3000)
        mine = shard.lpt_partition(sizes, world)[rank]
        x, m, off = synth.batch_subset(n_sys, seed, mine, 100, 3000)
        got = [None] * world
        dist.all_gather_object(got, (mine.tolist(), x.shape[0], float(m.sum()), float(np.abs(x).sum())))
        if rank == 0:
            out.put(got)
    finally:
        dist.destroy_process_group()


def test_sharded_batch_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world, n_sys, seed = 2, 24, 77
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n_sys, seed, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = out.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    idx = sorted(i for g in got for i in g[0])
    assert idx == list(range(n_sys))                      # every system exactly once
    assert not set(got[0][0]) & set(got[1][0])
    x, m, off = synth.batch(n_sys, seed, 100, 3000)
    assert sum(g[1] for g in got) == x.shape[0]          # the particles of the full batch
    assert np.isclose(sum(g[2] for g in got), m.sum(), rtol=1e-12)
    assert np.isclose(sum(g[3] for g in got), np.abs(x).sum(), rtol=1e-12)
    sizes = np.diff(off)
    cost = [shard.system_cost(sizes[np.array(g[0])]).sum() for g in got]
    assert max(cost) - min(cost) <= shard.system_cost(sizes).max()
