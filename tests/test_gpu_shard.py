"""perch_best_key on the GPU: the packed (J << 32 | id) key of each shard's
winner; the smallest key over the shards is the single-search argmin (the
value bench.py's all-reduce MIN combines across ranks)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_shard_keys_combine_to_the_whole_argmin():
    import torch
    from paper_2008_00326_gb300 import build, perch as P, shard
    build.build()
    rng = np.random.default_rng(12)
    with P.Context(0) as ctx:
        for n, world, hi in ((29584, 2, 40), (88752, 3, 3), (4097, 8, 100000), (5, 8, 2)):
            costs = rng.integers(0, hi, size=(n, 2)).astype(np.int32)
            want_i, want_j = ctx.best(costs)
            s = torch.cuda.Stream()
            keys = []
            for r in range(world):
                a, b = shard.shard_bounds(n, r, world)
                if b == a:
                    keys.append(shard.EMPTY_KEY)
                    continue
                dc = torch.from_numpy(costs[a:b]).cuda()
                ids = torch.arange(a, b, dtype=torch.int64, device="cuda")
                k = torch.full((1,), -1, dtype=torch.int64, device="cuda")
                with torch.cuda.stream(s):
                    P.perch_best_key(ctx.ctx, dc, k, ids=ids, stream=s)
                s.synchronize()
                keys.append(int(k.item()))
                # one shard alone: the key is its own argmin, packed
                li, lj = ctx.best(costs[a:b])
                assert shard.unpack(keys[-1]) == (lj, a + li)
            assert shard.unpack(min(keys)) == (want_j, want_i), (n, world)
