"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks.

Each rank owns a disjoint part of the k-mer space (owner-computes, Section 5.1), so the only
cross-rank operations are the timing barrier, the max over ranks and the sum of the windows
each rank counted. These tests run those helpers with gloo, and check with the oracle that
the owner partition makes per-rank results disjoint and complete."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ws, r, local = bench.dist_env()
        assert (ws, r, local) == (world, rank, rank)
        bench.barrier(ws)
        t = bench.max_over_ranks(10.0 + rank, ws)   # per-rank step times
        n = torch.tensor([100 + rank], dtype=torch.int64)
        dist.all_reduce(n)
        q.put((rank, t, int(n.item())))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_timing_and_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [11.0, 11.0]      # max over ranks
    assert [g[2] for g in got] == [201, 201]        # whole-job units


def test_owner_partitions_are_disjoint_and_complete():
    """The sharded path's correctness argument on the oracle: union over owners = whole."""
    import oracle
    import synth
    rs = synth.workload("plain_1m", scale=0.05)
    whole = oracle.run_readset(rs)
    parts = [oracle.run_readset(rs, part=i, n_parts=2) for i in range(2)]
    assert len(parts[0]) + len(parts[1]) == len(whole)
    keys = np.concatenate([p.keys for p in parts])
    assert len({(int(a), int(b)) for a, b in keys}) == len(whole)


def test_sizing_splits_across_owners():
    import bench
    import synth
    rs = synth.workload("plain_1m", scale=0.05)
    one = bench.workload_sizing(rs, 1)
    four = bench.workload_sizing(rs, 4)
    assert four["expected_keys"] < one["expected_keys"] / 3
    assert four["expected_distinct"] < one["expected_distinct"] / 3
