"""Pins for the oracle's 2-opt (Sec. 5.7: Bentley's neighbour-list 2-opt with
don't-look bits, first improvement)."""
import numpy as np
import pytest

import oracle as O
from paper_2003_11902_gb300 import instances as I


def _exchange(tour, i, j):
    """The tour after removing edges (t[i], t[i+1]) and (t[j], t[j+1]) and
    reconnecting t[i]-t[j], t[i+1]-t[j+1] (reverse t[i+1..j])."""
    t = list(tour)
    i, j = sorted((i, j))
    return np.array(t[:i + 1] + t[i + 1:j + 1][::-1] + t[j + 1:], dtype=np.int32)


def _improving_move_left(d, nn, tour):
    """Any move the neighbour-list rule admits (c2 in nn[c1] closer to c1 than
    c1's tour neighbour on that side) that shortens the tour, by performing it."""
    n = len(tour)
    pos = np.empty(n, int)
    pos[tour] = np.arange(n)
    base = O.tour_length(d, tour)
    for c1 in range(n):
        for side in (1, -1):
            nb = tour[(pos[c1] + side) % n]
            for c2 in nn[c1]:
                if d[c1, c2] >= d[c1, nb]:
                    break
                if side == 1:
                    i, j = pos[c1], pos[c2]        # remove (c1, s1) and (c2, s2)
                else:
                    i, j = (pos[c1] - 1) % n, (pos[c2] - 1) % n  # remove (p1, c1), (p2, c2)
                if i == j:
                    continue
                if O.tour_length(d, _exchange(tour, i, j)) < base:
                    return (c1, int(c2), side)
    return None


@pytest.mark.parametrize("kind,n,k,seed", [("uniform", 200, 8, 1), ("uniform", 300, 16, 2),
                                            ("clustered", 400, 16, 3)])
def test_two_opt_reaches_a_neighbour_list_local_optimum(kind, n, k, seed):
    xy = I.uniform(n, seed) if kind == "uniform" else I.clustered(n, seed)
    d = O.distances(xy)
    nn = O.candidates(d, k)
    start = I.random_permutation(n, seed + 10)
    tour, moves = O.two_opt(d, nn, start)
    assert np.array_equal(np.sort(tour), np.arange(n))
    assert moves > 0
    assert O.tour_length(d, tour) < O.tour_length(d, start)
    assert _improving_move_left(d, nn, tour) is None
    # a local optimum is a fixed point
    again, moves2 = O.two_opt(d, nn, tour)
    assert moves2 == 0 and np.array_equal(again, tour)


def test_two_opt_on_convex_points_reaches_the_hull():
    xy = I.convex(40, 8)
    d = O.distances(xy)
    nn = O.candidates(d, 39)
    c = xy - xy.mean(axis=0)
    hull = np.argsort(np.arctan2(c[:, 1], c[:, 0]))
    for s in range(5):
        tour, _ = O.two_opt(d, nn, I.random_permutation(40, 100 + s))
        assert O.tour_length(d, tour) == O.tour_length(d, hull)


def test_two_opt_untangles_a_crossed_square():
    xy = np.array([[0, 0], [10, 0], [10, 10], [0, 10]], np.int32)
    d = O.distances(xy)
    nn = O.candidates(d, 3)
    tour, moves = O.two_opt(d, nn, np.array([0, 2, 1, 3], np.int32))
    assert moves == 1 and O.tour_length(d, tour) == 40


@pytest.mark.parametrize("ls", [1, 2])
def test_colony_local_search_modes(ls):
    n, m = 60, 12
    xy = I.uniform(n, 71)
    plain = O.Colony(xy=xy, m=m, cl=8, rho=0.1, seed=4)
    col = O.Colony(xy=xy, m=m, cl=8, rho=0.1, seed=4, ls=ls)
    d = col.state()["d"]
    nn = col.state()["cand"]
    plain.iterate(1)
    col.iterate(1)
    ptours, plens, _ = plain.tours()
    tours, lens, _ = col.tours()
    # same construction; local search then improves the iteration best (ls = 1)
    # or every tour (ls = 2) to a neighbour-list local optimum
    ib = int(np.argmin(plens))
    for k in range(m):
        if ls == 2 or k == ib:
            want, _ = O.two_opt(d, nn, ptours[k])
            assert np.array_equal(tours[k], want)
            assert lens[k] == O.tour_length(d, want) <= plens[k]
        else:
            assert np.array_equal(tours[k], ptours[k])
    assert col.best()[0] == lens.min()
