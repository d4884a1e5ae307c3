"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own copy
of the batch (weak scaling); the reported step time is the slowest rank's and
the rate counts every rank's hypotheses."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0][rank]
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    rate = bench.whole_job_rate(88752, world, ms)
    q.put((rank, ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, rate in got:
        assert ms == 150.0
        assert rate == pytest.approx(2 * 88752 / 0.150)


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.whole_job_rate(1000, 1, 500.0) == 2000.0


# ---- the sharded search: each rank's share reduced to one packed key per
# object, then one min-reduce over the ranks


def _shard_rank(rank, world, port, q, costs_list):
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_2008_00326_gb300 import shard
    keys = []
    for costs in costs_list:
        a, b = shard.shard_bounds(len(costs), rank, world)
        if b > a:
            # the local argmin over this rank's share, ids = global indices
            bi, bc = O.best(costs[a:b], ids=np.arange(a, b, dtype=np.uint64))
            keys.append(shard.pack(bc, a + bi))
        else:
            keys.append(shard.EMPTY_KEY)
    t = torch.tensor(keys, dtype=torch.int64)
    shard.reduce_keys(t, dist)
    q.put((rank, [shard.unpack(int(k)) for k in t]))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_search_winner_equals_the_single_rank_argmin():
    """Two gloo ranks split each object's hypotheses; the min-reduced key is
    the single-rank argmin of all of them -- including ties that straddle the
    shards (lowest id wins) and an object too small to reach every rank."""
    import numpy as np
    import torch.multiprocessing as mp
    from oracle import oracle as O
    rng = np.random.default_rng(8)
    costs_list = [rng.integers(0, 40, size=(29584, 2)).astype(np.int32),    # many ties
                  rng.integers(0, 10_000, size=(4097, 2)).astype(np.int32),
                  np.full((1, 2), 3, np.int32)]                              # rank 1 gets nothing
    tie = costs_list[0].copy()
    tie[:] = 50
    tie[20000] = tie[7] = (0, 1)            # equal minima in both shards: id 7 wins
    costs_list.append(tie)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q, costs_list)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    want = []
    for costs in costs_list:
        bi, bc = O.best(costs)
        want.append((bc, bi))
    assert got[0] == want and got[1] == want
    assert want[3] == (1, 7)


def test_shard_bounds_cover_every_hypothesis_once():
    from paper_2008_00326_gb300 import shard
    for n in (0, 1, 7, 29584, 88752):
        for world in (1, 2, 3, 8):
            spans = [shard.shard_bounds(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1
    assert shard.unpack(shard.pack(123, 4567)) == (123, 4567)
    assert shard.pack(1, 0) > shard.pack(0, (1 << 32) - 1)       # the cost decides first
