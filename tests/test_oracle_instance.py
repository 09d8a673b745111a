"""Pins for the oracle's instance set-up: distances, heuristic weights,
candidate lists, the nearest-neighbour tour and the trail limits."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2003_11902_gb300 import instances as I


def test_isqrt_matches_python_exact_isqrt():
    rng = np.random.Generator(np.random.PCG64(1))
    vals = [0, 1, 2, 3, 4, 15, 16, 17, 2 ** 32 - 1, 2 ** 32, 2 ** 52 + 1, 2 ** 62 - 1, 2 ** 63]
    vals += [int(x) for x in rng.integers(0, 2 ** 63, size=2000, dtype=np.int64)]
    for s in vals:
        assert O.isqrt64(s) == math.isqrt(s)
    for q in [1, 2, 1000, 46340, 3037000499]:
        assert O.isqrt64(q * q) == q and O.isqrt64(q * q - 1) == q - 1


def test_euc2d_known_values():
    assert O.euc2d(0, 0, 3, 4) == 5
    assert O.euc2d(0, 0, 1, 1) == 1          # 1.414 -> 1
    assert O.euc2d(0, 0, 1, 2) == 2          # 2.236 -> 2
    assert O.euc2d(0, 0, 2, 3) == 4          # 3.606 -> 4
    assert O.euc2d(5, 5, 5, 5) == 0
    assert O.euc2d(0, 0, 99999, 99999) == 141420  # 141419.99 -> 141420


def test_euc2d_matches_double_nint_where_double_is_exact():
    rng = np.random.Generator(np.random.PCG64(2))
    p = rng.integers(-(2 ** 24), 2 ** 24, size=(5000, 4))
    for x1, y1, x2, y2 in p:
        s = float((x1 - x2) ** 2 + (y1 - y2) ** 2)  # < 2^51: exact in double
        assert O.euc2d(int(x1), int(y1), int(x2), int(y2)) == int(math.floor(math.sqrt(s) + 0.5))


def test_distance_matrix_properties():
    xy = I.uniform(60, 11)
    d = O.distances(xy)
    assert d.dtype == np.int32
    assert np.array_equal(d, d.T)
    assert np.all(np.diag(d) == 0)
    off = d[~np.eye(60, dtype=bool)]
    assert off.min() >= 1  # distinct points are at least 1 apart once rounded
    i, j = 3, 41
    assert d[i, j] == round(math.dist(xy[i], xy[j]))


def test_eta_beta_special_cases():
    xy = I.uniform(40, 12)
    d = O.distances(xy)
    off = ~np.eye(40, dtype=bool)
    e0 = O.eta_beta(d, 0.0)
    assert np.all(e0[off] == 1.0) and np.all(np.diag(e0) == 0.0)
    e1 = O.eta_beta(d, 1.0)
    assert np.array_equal(e1[off], (1.0 / d[off].astype(np.float64)).astype(np.float32))
    e2 = O.eta_beta(d, 2.0)
    ref = (1.0 / d[off].astype(np.float64) ** 2).astype(np.float32)
    np.testing.assert_allclose(e2[off], ref, rtol=1.2e-7, atol=0)


def test_eta_clamps_zero_distance():
    d = np.array([[0, 0, 5], [0, 0, 3], [5, 3, 0]], dtype=np.int32)
    eb = O.eta_beta(d, 2.0)
    assert eb[0, 1] == 1.0 and eb[1, 0] == 1.0
    assert eb[0, 0] == 0.0


def test_candidate_lists_match_lexsort():
    xy = I.grid(7, 6, spacing=10)  # many equal distances: exercises the id tie-break
    d = O.distances(xy)
    n = d.shape[0]
    cl = 9
    cand = O.candidates(d, cl)
    for i in range(n):
        j = np.array([x for x in range(n) if x != i])
        order = j[np.lexsort((j, d[i, j]))]
        assert np.array_equal(cand[i], order[:cl])


def test_nn_tour_on_a_line_closed_form():
    # points on a line, node 0 at the left end: the nearest-neighbour walk goes
    # right one point at a time, so the tour length is twice the span.
    xs = np.array([0, 3, 7, 8, 20, 21, 40, 66], dtype=np.int32)
    xy = np.stack([xs, np.zeros_like(xs)], axis=1)
    perm = np.array([0, 5, 2, 7, 1, 6, 3, 4])
    inv = np.argsort(perm)
    length, tour = O.nn_tour(O.distances(xy[perm]))
    assert length == 2 * 66
    assert np.array_equal(perm[tour], np.arange(8))
    assert tour[0] == 0 and inv[0] == 0


def test_nn_tour_tie_goes_to_lower_id():
    # node 0 in the middle, nodes 1 and 2 at equal distance: 1 is taken first
    xy = np.array([[10, 0], [20, 0], [0, 0], [30, 0]], dtype=np.int32)
    _, tour = O.nn_tour(O.distances(xy))
    assert list(tour) == [0, 1, 3, 2]


def test_tour_length_square():
    xy = np.array([[0, 0], [10, 0], [10, 10], [0, 10]], dtype=np.int32)
    d = O.distances(xy)
    assert O.tour_length(d, [0, 1, 2, 3]) == 40
    assert O.tour_length(d, [0, 2, 1, 3]) == 10 + 10 + 14 + 14


@pytest.mark.parametrize("n,rho,cost,p_best", [(10, 0.02, 100, 0.01), (1000, 0.02, 290032, 0.01),
                                               (200, 0.5, 31000, 0.05), (3, 0.1, 17, 0.01)])
def test_limits_defining_properties(n, rho, cost, p_best):
    tmax, tmin = O.limits(n, rho, p_best, cost)
    # tau_max is the fixed point of tau <- (1 - rho) tau + 1/C
    assert abs(float(tmax) * rho * cost - 1.0) < 1e-6
    assert 0 < tmin <= tmax
    # p_best is the chance of picking the best edge at each of n decisions when
    # it carries tau_max and the (n/2 - 1) other choices carry tau_min
    avg = n / 2.0
    if tmin < tmax:
        p_dec = float(tmax) / (float(tmax) + (avg - 1.0) * float(tmin))
        assert abs(p_dec ** n / p_best - 1.0) < 1e-4
