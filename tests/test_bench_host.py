"""Host logic of bench.py without a GPU: the algorithmic byte count behind the
roofline, the stored L* each time-to-2% figure reads, and the bookkeeping of
the time-to-2% runs, driven by stand-in colonies whose best length is a known
function of the iteration."""
import os

import numpy as np
import pytest

import bench


def test_algorithmic_construct_bytes():
    # the method's logical reads: per step each candidate's 4-byte weight and
    # 4-byte id, 256 B at cl = 32 -- 255.7 MB a launch at n = m = 1000 (the
    # figure of the survey's n = 1000 row: 256 B per step)
    w = bench.WORKLOADS["uniform-n1000-cl32"]
    assert bench.algorithmic_construct_bytes(w) == 1000 * 999 * 32 * 8 == 255_744_000
    # the clustered workload: 128 B per step, 3,800 - 1 steps per ant, 1000 ants
    w = bench.WORKLOADS["clustered-n3800-cl16-2opt"]
    assert bench.algorithmic_construct_bytes(w) == 1000 * 3799 * 16 * 8
    # whole rows: the unvisited weights of every step, 4 B each: n(n-1)/2 per ant
    w = bench.WORKLOADS["uniform-n200-fullrow"]
    assert bench.algorithmic_construct_bytes(w) == 200 * (4 * (200 * 199 // 2))
    # as stored: 16-bit ids and 4-byte reciprocal weights, plus the tour entries
    w = bench.WORKLOADS["uniform-n1000-cl32"]
    assert bench.stored_construct_bytes(w) == 1000 * (999 * 32 * 6 + 4 * 1000) == 195_808_000


def test_every_stored_lstar_exists():
    for wl, (fname, _) in bench.LSTAR_FILES.items():
        assert wl in bench.WORKLOADS
        assert os.path.exists(os.path.join(bench.ROOT, "tests", "golden", fname)), fname
    assert os.path.exists(os.path.join(bench.ROOT, "tests", "golden", "lstar_batched_sample16.json"))


class _FakeColony:
    """best length = 10^6 / (1 + iterations), or never below 10^9 when the seed is a multiple of 7."""

    def __init__(self, xy=None, seed=0, **kw):
        self.seed, self.it = seed, 0

    def iterate(self, k):
        self.it += k

    def best(self):
        return 10**9 if self.seed % 7 == 0 else 10**6 // (1 + self.it)

    def stats(self):
        return {"best_len": self.best()}

    def close(self):
        pass


class _FakeBatch:
    def __init__(self, xys=None, seed=0, **kw):
        self.cols = [_FakeColony(seed=seed + b) for b in range(len(xys))]

    def iterate(self, k):
        for c in self.cols:
            c.iterate(k)

    def best_lengths(self):
        return np.array([c.best() for c in self.cols])

    def close(self):
        pass


@pytest.fixture
def fakes(monkeypatch):
    import torch

    import paper_2003_11902_gb300 as P
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(P, "Colony", _FakeColony)
    monkeypatch.setattr(P, "Batch", _FakeBatch)


def test_batched_time_to_gap_bookkeeping(fakes):
    r = bench.batch_time_to_gap(bench.WORKLOADS["batched-256-n100-2000-cl32"], 1, 0, 0, max_iters=200)
    seeds = [1 + b for b in range(16)]
    never = [s % 7 == 0 for s in seeds]
    assert r["reached"] == 16 - sum(never) and r["max_iterations"] == 200
    # the same colonies reach the target after the same iterations both ways,
    # at the first multiple of 5 where 10^6 / (1 + it) <= 1.02 L*
    assert r["same_iterations"] and r["batch_iterations"] == r["single_iterations"]
    import json
    with open(os.path.join(bench.ROOT, "tests", "golden", "lstar_batched_sample16.json")) as f:
        lstar = [e["lstar"] for e in json.load(f)["instances"]]
    for b, it in enumerate(r["batch_iterations"]):
        if never[b]:
            assert it is None
        else:
            want = next(k for k in range(5, 201, 5) if 10**6 // (1 + k) <= 1.02 * lstar[b])
            assert it == want
    assert r["batch_seconds"] > 0 and r["single_seconds_total"] > 0
    assert r["speedup"] == pytest.approx(r["single_seconds_total"] / r["batch_seconds"])


def test_single_time_to_gap_reads_the_workload_lstar(fakes):
    w = bench.WORKLOADS["clustered-n3800-cl16-2opt"]
    r = bench.time_to_gap("clustered-n3800-cl16-2opt", w, None, 3, 0, 0, max_iters=100)
    assert r["lstar"] == 832831 and "lstar_clustered_n3800.json" in r["lstar_source"]
    # the stand-in's 10^6 / 6 is already within 2% of L* at the first check
    assert r["iterations"] == 5 and r["seconds"] is not None and r["target"] == 1.02 * 832831
    assert bench.time_to_gap("uniform-n200-fullrow", bench.WORKLOADS["uniform-n200-fullrow"], None, 3, 0, 0) is None
