"""The multi-rank protocol (ants sharded over ranks, one exchange per
iteration) on CPU ranks with the gloo backend, and the GPU side of it
(``ant_offset``) on one GPU.  The oracle builds each rank's shard; the run must
equal the single-colony run exactly."""
import os
import socket

import numpy as np
import pytest

from paper_2003_11902_gb300 import sharded
from paper_2003_11902_gb300 import instances as I


def test_shard_ranges_cover_the_colony():
    for m in (1, 7, 10, 1000):
        for world in (1, 2, 3, 4):
            seen = []
            for r in range(world):
                off, cnt = sharded.shard_range(m, r, world)
                seen.extend(range(off, off + cnt))
                for a in range(off, off + cnt):
                    assert sharded.owner_of(a, m, world) == r
            assert seen == list(range(m))
    assert sharded.unpack(sharded.pack(123456, 789)) == (123456, 789)
    assert sharded.pack(10, 5) < sharded.pack(10, 6) < sharded.pack(11, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, n, m, iters, out):
    import torch.distributed as dist

    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    xy = I.uniform(n, 55)
    col = O.Colony(xy=xy, m=m, cl=6, rho=0.2, seed=9)
    off, cnt = sharded.shard_range(m, rank, world)
    for it in range(iters):
        tours = np.zeros((cnt, n), np.int32)
        lens = np.zeros(cnt, np.int64)
        for i in range(cnt):
            lens[i], tours[i], _ = col.construct(it, off + i)
        length, ant, tour = sharded.exchange_iteration_best(lens, tours, off, m)
        col.update(tour, length)
    best_len, best_tour = col.best()
    np.save(out.format(rank=rank), np.concatenate([[best_len], best_tour]).astype(np.int64))
    np.save(out.format(rank=rank) + ".tau.npy", col.state()["tau"])
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_protocol_equals_one_colony(tmp_path, world):
    import torch.multiprocessing as mp

    import oracle as O
    n, m, iters = 30, 10, 6
    out = str(tmp_path / "rank{rank}.npy")
    mp.start_processes(_rank_main, args=(world, _free_port(), n, m, iters, out), nprocs=world,
                       start_method="spawn")
    ref = O.Colony(xy=I.uniform(n, 55), m=m, cl=6, rho=0.2, seed=9)
    ref.iterate(iters)
    ref_len, ref_tour = ref.best()
    ref_tau = ref.state()["tau"]
    for r in range(world):
        got = np.load(out.format(rank=r))
        assert got[0] == ref_len and np.array_equal(got[1:], ref_tour)
        assert np.array_equal(np.load(out.format(rank=r) + ".tau.npy"), ref_tau)


@pytest.mark.gpu
def test_gpu_shard_builds_the_same_ants():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_11902_gb300 import Colony
    xy = I.uniform(400, 3)
    whole = Colony(xy=xy, m=64, cl=16, seed=2)
    part = Colony(xy=xy, m=24, cl=16, seed=2, ant_offset=40)
    whole.construct()
    part.construct()
    wt, wl = whole.tours()
    pt, pl = part.tours()
    assert np.array_equal(wt[40:], pt) and np.array_equal(wl[40:], pl)
    whole.close()
    part.close()


class _OracleShard:
    """Host stand-in for a sharded GPU colony with the four methods the
    device-side exchange drives (construct, shard_best_key, shard_tour,
    update_device), on torch CPU tensors; its tours come from the oracle."""

    def __init__(self, xy, m, off, cnt, **kw):
        import oracle as O
        self.col = O.Colony(xy=xy, m=m, **kw)
        self.off, self.cnt, self.n = off, cnt, xy.shape[0]
        self.it = 0

    def construct(self):
        self.tours = np.zeros((self.cnt, self.n), np.int32)
        self.lens = np.zeros(self.cnt, np.int64)
        for i in range(self.cnt):
            self.lens[i], self.tours[i], _ = self.col.construct(self.it, self.off + i)

    def shard_best_key(self, key):
        k = int(np.argmin(self.lens))
        key[0] = sharded.pack(self.lens[k], self.off + k)

    def shard_tour(self, key, tour):
        ant = sharded.unpack(int(key[0]))[1]
        tour[:] = 0
        if self.off <= ant < self.off + self.cnt:
            tour[:] = __import__("torch").from_numpy(self.tours[ant - self.off])

    def update_device(self, tour, key):
        self.col.update(tour.numpy(), sharded.unpack(int(key[0]))[0])
        self.it += 1


def _rank_main_device(rank, world, port, n, m, iters, out):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    xy = I.uniform(n, 56)
    off, cnt = sharded.shard_range(m, rank, world)
    shard = _OracleShard(xy, m, off, cnt, cl=6, rho=0.2, seed=10)
    key = torch.zeros(1, dtype=torch.int64)
    tour = torch.zeros(n, dtype=torch.int32)
    sent = []
    rmin, rsum = sharded.nccl_reducers()

    def count(f):
        def g(t):
            sent.append(t.numel() * t.element_size())
            f(t)
        return g
    for _ in range(iters):
        sharded.sharded_iteration_device(shard, key, tour, count(rmin), count(rsum))
    best_len, best_tour = shard.col.best()
    np.save(out.format(rank=rank), np.concatenate([[best_len], best_tour, sent]).astype(np.int64))
    np.save(out.format(rank=rank) + ".tau.npy", shard.col.state()["tau"])
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_device_side_exchange_protocol_equals_one_colony(tmp_path, world):
    # the exchange driven as on the GPU (key MIN, owner-filled tour SUM, update
    # from the reduced buffers), here on host tensors over gloo: equal to one
    # colony, and 8 + 4n bytes cross ranks per iteration
    import torch.multiprocessing as mp

    import oracle as O
    n, m, iters = 30, 10, 6
    out = str(tmp_path / "rank{rank}.npy")
    mp.start_processes(_rank_main_device, args=(world, _free_port(), n, m, iters, out), nprocs=world,
                       start_method="spawn")
    ref = O.Colony(xy=I.uniform(n, 56), m=m, cl=6, rho=0.2, seed=10)
    ref.iterate(iters)
    ref_len, ref_tour = ref.best()
    for r in range(world):
        got = np.load(out.format(rank=r))
        assert got[0] == ref_len and np.array_equal(got[1:n + 1], ref_tour)
        sent = got[n + 1:].reshape(iters, 2)
        assert np.all(sent[:, 0] == 8) and np.all(sent[:, 1] == 4 * n)
        assert np.array_equal(np.load(out.format(rank=r) + ".tau.npy"), ref.state()["tau"])


@pytest.mark.gpu
def test_gpu_device_side_exchange_equals_one_colony():
    # three shards of one colony on one GPU, their all-reduces done by tensor
    # operations on the device: tours, best and pheromone equal the single
    # colony's after every iteration, with no host copy inside the loop
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_11902_gb300 import Colony
    n, m, iters, world = 500, 90, 8, 3
    xy = I.uniform(n, 4)
    whole = Colony(xy=xy, m=m, cl=16, seed=5)
    shards = [Colony(xy=xy, m=sharded.shard_range(m, r, world)[1], cl=16, seed=5,
                     ant_offset=sharded.shard_range(m, r, world)[0]) for r in range(world)]
    keys = [torch.zeros(1, dtype=torch.int64, device="cuda") for _ in range(world)]
    tours = [torch.zeros(n, dtype=torch.int32, device="cuda") for _ in range(world)]

    for it in range(iters):
        for c in shards:
            c.construct()
        for c, k in zip(shards, keys):
            c.shard_best_key(k)
        kmin = torch.stack(keys).min(dim=0).values
        for k in keys:
            k.copy_(kmin)
        for c, k, t in zip(shards, keys, tours):
            c.shard_tour(k, t)
        tsum = torch.stack(tours).sum(dim=0).to(torch.int32)
        for t in tours:
            t.copy_(tsum)
        for c, t, k in zip(shards, tours, keys):
            c.update_device(t, k)
        whole.iterate(1)
        wt, wl = whole.tours()
        lo = 0
        for c in shards:
            st, sl = c.tours()
            assert np.array_equal(wt[lo:lo + c.m], st) and np.array_equal(wl[lo:lo + c.m], sl)
            lo += c.m
    wlen, wtour = whole.best_tour()
    wtau = whole.pheromone()
    for c in shards:
        blen, btour = c.best_tour()
        assert blen == wlen and np.array_equal(btour, wtour)
        tau = c.pheromone()
        assert np.array_equal(tau[0], wtau[0]) and tau[1:] == wtau[1:]
        assert c.stats()["iterations"] == iters
        c.close()
    # a buffer that is not a permutation is refused on the device
    bad = torch.zeros(n, dtype=torch.int32, device="cuda")
    whole.update_device(bad, keys[0])
    with pytest.raises(Exception, match="not a permutation"):
        whole.synchronize()
    whole.close()
