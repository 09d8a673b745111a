"""Batched colonies (one construction, one scoring and one pheromone launch per
iteration for every colony) against the oracle and against single colonies.

Colony b of a batch must equal the colony built from instance b alone with seed
+ b: the same tours, lengths, best tour and pheromone, iteration by iteration,
whatever the launch shape of the batched construction."""
import numpy as np
import pytest

import oracle as O
from paper_2003_11902_gb300 import Batch, Colony, MMASError, instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


# sizes spanning: register tabu + staged table, n > 1024 (shared-memory tabu),
# a table too large to stage (n = 2000, cl = 32: 375 KB), ragged n
SIZES = [37, 300, 700, 1100, 2000, 129]


def _oracle(xy, m, cl, rho, seed):
    return O.Colony(xy=xy, m=m, cl=cl, rho=rho, seed=seed, p_best=float(np.float32(0.01)))


def test_batch_colonies_match_the_oracle():
    xys = [I.uniform(n, 900 + n) for n in SIZES]
    m, cl, rho, seed = 24, 32, 0.1, 11  # cl <= min(n) - 1 = 36
    bt = Batch(xys=xys, m=m, cl=cl, rho=rho, seed=seed)
    orcs = [_oracle(xy, m, cl, rho, seed + b) for b, xy in enumerate(xys)]
    for it in range(3):
        bt.iterate(1)
        for b, o in enumerate(orcs):
            o.iterate(1)
            tours, lens = bt.tours(b)
            ot, ol, _ = o.tours()
            assert np.array_equal(lens, ol), f"colony {b} (n={SIZES[b]}) iteration {it}: lengths"
            assert np.array_equal(tours, ot), f"colony {b} iteration {it}: tours"
            blen, btour = bt.best_tour(b)
            olen, otour = o.best()
            assert blen == olen and np.array_equal(btour, otour)
    assert list(bt.best_lengths()) == [o.best()[0] for o in orcs]
    bt.close()


@pytest.mark.parametrize("sizes,cfgs,cands", [
    # every colony n <= 2048: the 16-warp variant of the batched construction
    ((200, 1300, 64, 900), [(16, 1), (12, 1), (4, 3), (5, 2)],
     [(16, 1), (14, 1), (12, 1), (8, 2), (4, 4), (5, 3)]),
    # a colony above 2048 (four-word tabus): the 12-warp variant
    ((200, 2500, 64), [(12, 1), (4, 3)], [(12, 1), (8, 1), (6, 2), (4, 3), (3, 4), (10, 1)]),
])
def test_launch_shape_does_not_change_results(sizes, cfgs, cands):
    xys = [I.uniform(n, 700 + n) for n in sizes]
    runs = []
    for cfg in cfgs + [None]:
        bt = Batch(xys=xys, m=40, cl=16, rho=0.05, seed=3)
        if cfg is None:
            chosen = bt.autotune(reps=1)
            assert chosen in cands
            assert bt.fallback_steps() == 0  # autotuning leaves no trace in the counters
        else:
            bt.set_config(*cfg)
            assert bt.config() == cfg
        bt.iterate(4)
        runs.append([bt.tours(b) for b in range(len(xys))] + [tuple(bt.best_lengths())])
        bt.close()
    for r in runs[1:]:
        for a, b in zip(runs[0][:-1], r[:-1]):
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert runs[0][-1] == r[-1]


def test_batch_colony_equals_single_colony_at_full_size():
    xys = [I.uniform(n, 500 + n) for n in (1000, 450, 1500)]
    bt = Batch(xys=xys, m=0, cl=32, seed=21)  # m = n per colony
    bt.iterate(3)
    for b, xy in enumerate(xys):
        col = Colony(xy=xy, m=len(xy), cl=32, seed=21 + b)
        col.iterate(3)
        t1, l1 = bt.tours(b)
        t2, l2 = col.tours()
        assert np.array_equal(l1, l2) and np.array_equal(t1, t2)
        assert bt.best_tour(b)[0] == col.best_tour()[0]
        col.close()
    bt.close()


def test_batch_with_explicit_matrices():
    ds = [O.distances(I.uniform(n, 600 + n)) for n in (50, 90)]
    bt = Batch(dists=ds, m=16, cl=8, rho=0.1, seed=2)
    orcs = [O.Colony(dist=d, m=16, cl=8, rho=0.1, seed=2 + b, p_best=float(np.float32(0.01)))
            for b, d in enumerate(ds)]
    bt.iterate(2)
    for b, o in enumerate(orcs):
        o.iterate(2)
        t, lens = bt.tours(b)
        ot, ol, _ = o.tours()
        assert np.array_equal(lens, ol) and np.array_equal(t, ot)
    bt.close()


def test_batch_errors_and_timing():
    bt = Batch(xys=[I.uniform(60, 1), I.uniform(80, 2)], m=8, cl=8)
    with pytest.raises(MMASError, match="ESTATE"):
        bt.best_tour(0)
    assert list(bt.best_lengths()) == [-1, -1]
    from paper_2003_11902_gb300.mmas import MMAS_EINVAL, load
    assert load().mmas_batch_get_tours(bt._b, 2, None, None) == MMAS_EINVAL
    assert "out of range" in load().mmas_batch_last_error(bt._b).decode()
    with pytest.raises(MMASError, match="warps_per_cta"):
        bt.set_config(17, 1)
    with pytest.raises(MMASError, match="exceeds"):
        bt.set_config(9, 2)
    assert bt.config() == (16, 1)  # a rejected shape leaves the batch as it was
    bt.enable_phase_timing(True)
    bt.iterate(2)
    c, r, t = bt.phase_times()
    assert c > 0 and r > 0 and abs(t - c - r) < 1e-6
    assert all(x > 0 for x in bt.best_lengths())
    bt.close()


def test_batch_colony_handle_shares_state():
    from paper_2003_11902_gb300 import Prior
    xys = [I.uniform(n, 70 + n) for n in (150, 400, 90)]
    bt = Batch(xys=xys, m=16, cl=16, seed=3)
    bt.iterate(2)
    col = bt.colony(1)
    blen, btour = bt.best_tour(1)
    clen, ctour = col.best_tour()
    assert clen == blen and np.array_equal(ctour, btour)
    # an iteration on the handle advances the batch's colony 1 (and only it)
    before = bt.best_lengths()
    col.iterate(3)
    after = bt.best_lengths()
    assert after[1] == col.best_tour()[0] and after[1] <= before[1]
    assert after[0] == before[0] and after[2] == before[2]
    pr = Prior(I.prior_params(3))
    s = pr.scores(col)
    assert s.shape == (400, 16) and np.isfinite(s).all()
    pr.close()
    col.close()  # drops the reference only
    bt.iterate(1)
    assert (bt.best_lengths() > 0).all()
    with pytest.raises(MMASError):
        bt.colony(3)
    bt.close()
