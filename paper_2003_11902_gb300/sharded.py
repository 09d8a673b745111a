"""Sharding one colony's ants over ranks (one process per GPU).

Within an iteration the ants are independent given the pheromone (Sec. 2.1:
MMAS has no local pheromone update), so rank r builds ants
[offset_r, offset_r + m_r) of the whole colony (``ant_offset`` in the C ABI
keys the draws by the global ant index).  The iteration's single exchange is:

  1. an all-reduce (MIN) of the packed key (length << 32 | global ant), which
     selects the shortest tour with ties to the lower ant, as Alg. 1's
     iteration-best step does for one colony;
  2. a broadcast of that tour (n ids) from the rank that owns the ant.

Every rank then applies the same deterministic update to its replica of the
pheromone, so the replicas stay identical and the run equals the single-colony
run whatever the number of ranks.  The exchange is 8 + 4n bytes per iteration.

``sharded_iteration_device`` keeps the whole exchange on the GPU: the library
writes the packed key and the owner's tour into device buffers
(mmas_shard_best_key, mmas_shard_tour), the ranks all-reduce them (MIN, then
SUM of a buffer that only the owner fills), and mmas_update_device applies the
update from the device tour, with no host copy.  ``sharded_iteration`` is the
host-side form (tours copied out, argmin on the host, tour copied back).
"""
from __future__ import annotations

import numpy as np

__all__ = ["shard_range", "owner_of", "pack", "unpack", "exchange_iteration_best",
           "sharded_iteration", "sharded_iteration_device", "nccl_reducers"]


def shard_range(m: int, rank: int, world: int):
    """(offset, count) of rank's contiguous block of the m ants."""
    base, extra = divmod(m, world)
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def owner_of(ant: int, m: int, world: int) -> int:
    for r in range(world):
        off, cnt = shard_range(m, r, world)
        if off <= ant < off + cnt:
            return r
    raise ValueError("ant out of range")


def pack(length: int, ant: int) -> int:
    return (int(length) << 32) | int(ant)


def unpack(key: int):
    return int(key) >> 32, int(key) & 0xFFFFFFFF


def exchange_iteration_best(lens, tours, offset: int, m: int, group=None, device="cpu"):
    """All ranks: (length, global ant, tour) of the shortest tour over all shards.

    ``lens`` and ``tours`` are this rank's local lengths (m_r) and tours
    (m_r x n).  Uses torch.distributed (gloo on CPU, NCCL with ``device`` a GPU).
    """
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    lens = np.asarray(lens)
    k = int(np.argmin(lens))  # ties -> lower local index -> lower global ant
    key = torch.tensor([pack(lens[k], offset + k)], dtype=torch.int64, device=device)
    dist.all_reduce(key, op=dist.ReduceOp.MIN, group=group)
    length, ant = unpack(key.item())
    owner = owner_of(ant, m, world)
    n = np.asarray(tours).shape[1]
    if rank == owner:
        buf = torch.from_numpy(np.ascontiguousarray(tours[ant - offset], dtype=np.int32)).to(device)
    else:
        buf = torch.empty(n, dtype=torch.int32, device=device)
    dist.broadcast(buf, src=dist.get_global_rank(group, owner) if group is not None else owner,
                   group=group)
    return length, ant, buf.cpu().numpy()


def nccl_reducers(group=None):
    """The exchange's two all-reduces for torch.distributed (NCCL between GPUs,
    gloo on host tensors): MIN of the key, SUM of the tour buffer, in place."""
    import torch.distributed as dist

    def rmin(t):
        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)

    def rsum(t):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return rmin, rsum


def sharded_iteration_device(colony, key, tour, reduce_min, reduce_sum):
    """One iteration of a sharded colony with the exchange on device buffers:
    construct this shard's ants; key (1 int64) = its shortest tour's packed
    (length, global ant); all-reduce MIN; tour (n int32) = that ant's tour if
    this shard owns it, else zeros; all-reduce SUM; the common update, which
    advances the iteration.  Only key and tour cross ranks: 8 + 4n bytes.
    ``colony`` is a ``Colony`` built with this rank's m and ant_offset (or any
    object with the same four methods); nothing is copied to the host."""
    colony.construct()
    colony.shard_best_key(key)
    reduce_min(key)
    colony.shard_tour(key, tour)
    reduce_sum(tour)
    colony.update_device(tour, key)


def sharded_iteration(colony, it: int, m_total: int, group=None, device="cpu"):
    """One iteration of a sharded GPU colony (a ``Colony`` built with this
    rank's ``m`` and ``ant_offset``): build the shard's tours for iteration
    ``it``, exchange the iteration best, apply the common update."""
    colony.set_iteration(it)
    colony.construct()
    tours, lens = colony.tours()
    length, ant, tour = exchange_iteration_best(lens, tours, colony.ant_offset, m_total, group,
                                                device)
    colony.update(tour, length)
    return length, ant
