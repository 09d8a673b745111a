"""The stored long-run bests L* (tests/golden/lstar_*.json, written by
tests/golden/make_lstar.py from the oracle) against what fixes them
independently: the benchmark builds the same instances, every L* lies between
the 2-neighbour lower bound (each node is entered and left by one edge, each at
least as long as its nearest and second-nearest neighbour distances) and the
length of a simple constructive tour, and each file is consistent with itself."""
import json
import os
import sys

import numpy as np
import pytest

import bench
import oracle as O
from paper_2003_11902_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
import make_lstar  # noqa: E402

# stored file -> (generator workload, benchmark workload)
SINGLE = {"lstar_uniform_n1000.json": ("uniform-n1000", "uniform-n1000-cl32"),
          "lstar_uniform_n1000_cl16_2opt.json": ("uniform-n1000-cl16-2opt", "learned-prior-n1000-cl16-2opt"),
          "lstar_clustered_n3800.json": ("clustered-n3800", "clustered-n3800-cl16-2opt")}


def _load(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    with open(path) as f:
        return json.load(f)


def _two_nn_bound(d):
    """Sum over nodes of half their two shortest incident distances (a lower
    bound on every tour: each node has two tour edges)."""
    d = d.astype(np.float64) + np.diag(np.full(len(d), np.inf))
    two = np.sort(d, axis=1)[:, :2]
    return float(two.sum()) / 2.0


def _check_bounds(xy, lstar, ls):
    d = O.distances(xy)
    assert _two_nn_bound(d) <= lstar
    _, nn = O.nn_tour(d)
    upper = O.tour_length(d, nn)
    if ls:  # the 2-opt local optimum of the nearest-neighbour tour
        cand = O.candidates(d, 16)
        upper = O.tour_length(d, O.two_opt(d, cand, nn)[0])
    assert lstar < upper, (lstar, upper)


@pytest.mark.parametrize("name", sorted(SINGLE))
def test_single_colony_lstar(name):
    data = _load(name)
    gen, wl = SINGLE[name]
    g, w = make_lstar.WORKLOADS[gen], bench.WORKLOADS[wl]
    # the benchmark's workload is the instance and colony the oracle ran
    for key in ("n", "m", "cl", "iseed"):
        assert g[key] == w[key], key
    assert g["ls"] == w.get("ls", 0)
    xy = bench._instance(w)
    assert np.array_equal(xy, make_lstar.instance(g))
    assert bench.LSTAR_FILES[wl][0] == name
    assert data["iterations"] == g["iters"]
    runs = data["runs"]
    assert [r["seed"] for r in runs] == [1, 2, 3]
    assert data["lstar"] == min(r["best"] for r in runs)
    for r in runs:  # a global best never gets worse
        tr = r["trace_every_50"]
        assert all(a >= b for a, b in zip(tr, tr[1:])) and tr[-1] == r["best"]
    _check_bounds(xy, data["lstar"], g["ls"])


def test_batched_sample_lstar():
    data = _load(make_lstar.BATCH_SAMPLE["out"])
    w = bench.WORKLOADS["batched-256-n100-2000-cl32"]
    xys = bench._batch_instances(w)
    insts = data["instances"]
    assert [(e["index"], e["n"]) for e in insts] == make_lstar.batch_sample()
    assert len(insts) == 16 and all(e["n"] <= 400 for e in insts)
    assert data["iterations"] == make_lstar.BATCH_SAMPLE["iters"]
    for e in insts:
        xy = xys[e["index"]]
        assert len(xy) == e["n"]
        assert np.array_equal(xy, I.uniform(e["n"], 1000 + e["index"]))
        assert e["lstar"] == min(r["best"] for r in e["runs"])
        _check_bounds(xy, e["lstar"], 0)
