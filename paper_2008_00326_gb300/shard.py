"""A pose search sharded over several processes, one GPU each.

Hypotheses are independent problems (Sec. IV-A "Parallel Search"): every rank
keeps the whole scene and meshes resident and scores its own share of each
object's hypotheses; the only exchange is the per-object argmin.  Each rank
reduces its share to one 64-bit key, (J << 32) | global hypothesis id
(perch_best_key on the device), and one min-reduce of the keys over the ranks
gives the winner of the whole search -- smallest J, ties to the lowest id, the
same pose a single perch_best over every hypothesis returns.

Host logic only: the keys are made by the library's argmin kernel, the
reduction by torch.distributed (NCCL between GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

EMPTY_KEY = (1 << 63) - 1     # a rank with no hypotheses of an object: never the minimum


def shard_bounds(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous share [start, stop) of n hypotheses for `rank` of `world`:
    the first n % world ranks take one more."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard")
    q, r = divmod(n, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def pack(J: int, gid: int) -> int:
    """(J << 32) | gid for a cost 0 <= J < 2^31 and an id 0 <= gid < 2^32."""
    if not (0 <= J < (1 << 31)) or not (0 <= gid < (1 << 32)):
        raise ValueError("cost or id out of range for a packed key")
    return (J << 32) | gid


def unpack(key: int) -> tuple[int, int]:
    """(J, gid) of a packed key."""
    return key >> 32, key & 0xFFFFFFFF


def reduce_keys(keys, dist):
    """Min-reduce a 1-D int64 torch tensor of per-object keys over all ranks,
    in place (an all-reduce MIN); without a process group it is returned as
    it is."""
    if dist is None:
        return keys
    dist.all_reduce(keys, op=dist.ReduceOp.MIN)
    return keys
