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
