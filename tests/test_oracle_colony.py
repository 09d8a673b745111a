"""Pins for the oracle's MMAS main loop (Alg. 1): valid tours, lengths,
best-so-far bookkeeping, trail limits, invariants, and tour quality against
exact optima (brute force, convex position, a lattice)."""
import numpy as np
import pytest

import oracle as O
from paper_2003_11902_gb300 import instances as I


def _is_perm(t, n):
    return len(t) == n and np.array_equal(np.sort(t), np.arange(n))


@pytest.mark.parametrize("cl,fallback", [(0, 0), (5, 0), (5, 1)])
def test_iterations_keep_invariants(cl, fallback):
    n, m = 40, 20
    col = O.Colony(xy=I.uniform(n, 101), m=m, cl=cl, rho=0.1, seed=9, fallback=fallback)
    d = col.state()["d"]
    best_seen = None
    prev_best = None
    for it in range(15):
        col.iterate(1)
        tours, lens, _ = col.tours()
        for k in range(m):
            assert _is_perm(tours[k], n)
            assert lens[k] == O.tour_length(d, tours[k])
        best_seen = lens.min() if best_seen is None else min(best_seen, lens.min())
        bl, bt = col.best()
        assert bl == best_seen and O.tour_length(d, bt) == bl
        if prev_best is not None:
            assert bl <= prev_best
        prev_best = bl
        tmin, tmax = col.limits()
        want_tmax, want_tmin = O.limits(n, np.float32(0.1), 0.01, bl)
        assert (tmax, tmin) == (want_tmax, want_tmin)
        tau = col.state()["tau"]
        assert np.all(tau >= tmin) and np.all(tau <= tmax)
        assert np.array_equal(tau, tau.T)
    assert col.iteration == 15


def test_one_iteration_by_hand():
    # rebuild iteration 0 from the oracle's own primitives, in Alg. 1's order
    n, m, rho = 15, 6, 0.2
    xy = I.uniform(n, 202)
    col = O.Colony(xy=xy, m=m, cl=4, rho=rho, seed=4)
    st = col.state()
    tmin0, tmax0 = col.limits()
    assert np.all(st["tau"] == tmax0)
    nn_len, _ = O.nn_tour(st["d"])
    want_tmax, want_tmin = O.limits(n, np.float32(rho), 0.01, nn_len)
    assert tmax0 == want_tmax and tmin0 == want_tmin
    tours = []
    lens = []
    for k in range(m):
        L, t, _ = col.construct(0, k)
        tours.append(t)
        lens.append(L)
    col.iterate(1)
    got_tours, got_lens, _ = col.tours()
    assert np.array_equal(np.array(tours), got_tours) and list(got_lens) == lens
    ib = int(np.argmin(lens))
    tmax, tmin = O.limits(n, np.float32(rho), 0.01, lens[ib])
    tau = O.evaporate(st["tau"], O.persist_factor(rho), tmin, tmax)
    tau = O.deposit(tau, tours[ib], np.float32(1.0 / lens[ib]), tmax)
    after = col.state()
    assert np.array_equal(after["tau"], tau)
    assert np.array_equal(after["choice"], O.choice(tau, st["eta_beta"], 1.0))


def test_deterministic_and_thread_independent():
    xy = I.uniform(60, 303)
    a = O.Colony(xy=xy, m=16, cl=8, seed=12)
    b = O.Colony(xy=xy, m=16, cl=8, seed=12)
    a.iterate(3, threads=1)
    b.iterate(3, threads=4)
    assert np.array_equal(a.tours()[0], b.tours()[0])
    assert np.array_equal(a.state()["tau"], b.state()["tau"])
    c = O.Colony(xy=xy, m=16, cl=8, seed=13)
    c.iterate(3)
    assert not np.array_equal(a.tours()[0], c.tours()[0])


def test_global_best_deposit_variant():
    xy = I.uniform(30, 404)
    col = O.Colony(xy=xy, m=10, cl=6, seed=2, deposit=1, rho=0.3)
    st = col.state()
    col.iterate(2)
    bl, bt = col.best()
    # replay iteration 1 on top of iteration 0's pheromone
    col0 = O.Colony(xy=xy, m=10, cl=6, seed=2, deposit=1, rho=0.3)
    col0.iterate(1)
    tau0 = col0.state()["tau"]
    tmin, tmax = col.limits()
    tau = O.evaporate(tau0, O.persist_factor(0.3), tmin, tmax)
    tau = O.deposit(tau, bt, np.float32(1.0 / bl), tmax)
    assert np.array_equal(col.state()["tau"], tau)
    assert st is not None


def test_brute_force_on_convex_position():
    # for points in convex position the optimal tour is the hull order
    xy = I.convex(9, 55)
    d = O.distances(xy)
    c = xy - xy.mean(axis=0)
    hull = np.argsort(np.arctan2(c[:, 1], c[:, 0]))
    opt, tour = O.brute_force(d)
    assert opt == O.tour_length(d, hull)
    assert O.tour_length(d, tour) == opt and _is_perm(tour, 9)


def test_mmas_reaches_brute_force_optimum_small():
    for seed in (1, 2):
        xy = I.uniform(9, 500 + seed, side=1000)
        d = O.distances(xy)
        opt, _ = O.brute_force(d)
        col = O.Colony(xy=xy, m=9, cl=0, rho=0.1, seed=seed)
        for _ in range(60):
            col.iterate(1)
            _, lens, _ = col.tours()
            assert lens.min() >= opt
        assert col.best()[0] == opt


def test_mmas_on_a_lattice_reaches_the_closed_form_optimum():
    # an even lattice with spacing s has an optimal tour of n * s
    xy = I.grid(6, 6, spacing=100)
    n = 36
    col = O.Colony(xy=xy, m=36, cl=8, rho=0.1, seed=3)
    for _ in range(150):
        col.iterate(1)
        assert col.tours()[1].min() >= n * 100
    assert col.best()[0] == n * 100
