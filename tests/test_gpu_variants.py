"""Whole-row variants on the GPU (Sec. 4.1 compact tabu, Sec. 4.2.1 roulette
wheel) against the oracle, iteration by iteration in lockstep: every step of
every GPU tour is replayed by the oracle on the GPU's prefix (teacher forcing,
tests/parity.py).  Roulette picks may differ only where the draw lies within
the single-precision rounding bound of an interval boundary, reservoir picks
only at near-ties; lengths are bit-exact and the pheromone agrees within
1e-5 relative after the oracle applies the GPU's iteration best."""
import numpy as np
import pytest

import oracle as O
from paper_2003_11902_gb300 import Colony, instances as I
from parity import check_ant_variant

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("selection,tabu", [(1, 0), (1, 1), (0, 1)])
@pytest.mark.parametrize("n,m,iters", [(40, 20, 6), (200, 24, 3), (1300, 12, 1)])
def test_variant_matches_oracle(selection, tabu, n, m, iters):
    xy = I.uniform(n, 300 + n)
    kw = dict(m=m, cl=0, rho=0.1, seed=5, selection=selection, tabu=tabu)
    g = Colony(xy=xy, **kw)
    o = O.Colony(xy=xy, p_best=float(np.float32(0.01)), **kw)
    d = o.state()["d"]
    counts = {"steps": 0, "boundary": 0, "near_tie": 0}
    for it in range(iters):
        g.iterate(1)
        t, lens = g.tours()
        for k in range(m):
            check_ant_variant(o, it, k, t[k], counts)
            assert lens[k] == O.tour_length(d, t[k]), f"ant {k}: length"
        ib = int(np.argmin(lens))  # ties -> lower ant
        o.update(t[ib], int(lens[ib]))
        tau, tmin, tmax = g.pheromone()
        assert (tmin, tmax) == o.limits()
        np.testing.assert_allclose(tau, o.state()["tau"], rtol=1e-5, atol=0)
    print(f"selection {selection} tabu {tabu} n {n}: {counts['steps']} steps, "
          f"{counts['boundary']} near-boundary and {counts['near_tie']} near-tie divergences")
    assert counts["boundary"] + counts["near_tie"] <= counts["steps"] // 1000 + 1
    g.close()


def test_gpu_reservoir_runs_match_oracle_roulette_quality():
    # whole runs of the GPU's reservoir selection and of the oracle's
    # sequential roulette wheel both sample Eq. (1): over 20 seeds their final
    # best lengths are one distribution (rank-sum test)
    stats = pytest.importorskip("scipy.stats")
    n, iters = 60, 40
    xy = I.uniform(n, 4242)
    gpu, orc = [], []
    for seed in range(1, 21):
        g = Colony(xy=xy, m=n, cl=0, rho=0.1, seed=seed)
        g.iterate(iters)
        gpu.append(g.best_tour()[0])
        g.close()
        o = O.Colony(xy=xy, m=n, cl=0, rho=0.1, seed=seed, selection=1, p_best=float(np.float32(0.01)))
        o.iterate(iters, threads=1)
        orc.append(int(o.best()[0]))
    print(f"GPU reservoir mean {np.mean(gpu):.0f}, oracle roulette mean {np.mean(orc):.0f}")
    assert stats.mannwhitneyu(gpu, orc).pvalue > 1e-3
