"""Pins for the oracle's pheromone rules (Sec. 2.1, Alg. 1): evaporation with
the lower clamp, deposit on the tour edges with the upper clamp, choice_info."""
import numpy as np

import oracle as O
from paper_2003_11902_gb300 import instances as I


def test_choice_alpha_one_is_the_float_product():
    n = 50
    tau = I.random_pheromone(n, 1, 1e-4, 1e-2)
    eb = I.random_pheromone(n, 2, 1e-8, 1e-4)
    ch = O.choice(tau, eb, 1.0)
    assert np.array_equal(ch, tau * eb)  # numpy float32 product, correctly rounded


def test_choice_alpha_half():
    n = 30
    tau = I.random_pheromone(n, 3, 1e-4, 1e-2)
    eb = I.random_pheromone(n, 4, 1e-8, 1e-4)
    ch = O.choice(tau, eb, 0.5)
    ref = (np.sqrt(tau.astype(np.float64)) * eb).astype(np.float32)
    np.testing.assert_allclose(ch, ref, rtol=1.2e-7)


def test_evaporation_closed_form_without_deposit():
    n, rho = 20, 0.1
    tmax, tmin = O.limits(n, rho, 0.01, 500)
    persist = O.persist_factor(rho)
    tau = np.full((n, n), tmax, np.float32)
    for t in range(1, 80):
        tau = O.evaporate(tau, persist, tmin, tmax)
        want = max(float(tmax) * (1.0 - rho) ** t, float(tmin))
        np.testing.assert_allclose(tau, want, rtol=1e-5)
    # far past the crossing, every cell sits exactly on the floor
    for _ in range(200):
        tau = O.evaporate(tau, persist, tmin, tmax)
    assert np.all(tau == tmin)


def test_evaporation_is_the_float_product_then_clamp():
    n = 40
    tau = I.random_pheromone(n, 5, 1e-4, 1e-2)
    persist = O.persist_factor(0.02)
    tmin, tmax = np.float32(2e-4), np.float32(5e-3)
    got = O.evaporate(tau, persist, tmin, tmax)
    want = np.minimum(np.maximum(tau * persist, tmin), tmax)  # float32 ops
    assert np.array_equal(got, want)
    assert np.any(tau * persist > tmax) and np.any(tau * persist < tmin)


def test_deposit_touches_exactly_the_tour_edges_symmetrically():
    n = 25
    tau = I.random_pheromone(n, 6, 1e-4, 1e-3)
    tour = I.random_permutation(n, 7)
    delta, tmax = np.float32(1e-4), np.float32(5e-3)
    new = O.deposit(tau, tour, delta, tmax)
    edges = set()
    for t in range(n):
        a, b = int(tour[t]), int(tour[(t + 1) % n])
        edges.add((a, b))
        edges.add((b, a))
    changed = set(zip(*np.nonzero(new != tau)))
    assert changed == edges and len(edges) == 2 * n
    for (a, b) in edges:
        assert new[a, b] == min(np.float32(tau[a, b] + delta), tmax)
    assert np.array_equal(new, new.T)


def test_deposit_clamps_at_tau_max():
    n = 5
    tau = np.full((n, n), 0.9, np.float32)
    new = O.deposit(tau, np.arange(n), np.float32(0.5), np.float32(1.0))
    assert new[0, 1] == 1.0 and new[4, 0] == 1.0 and new[0, 2] == np.float32(0.9)


def test_repeated_update_converges_to_the_limits():
    # an edge reinforced every iteration by 1/C tends to 1/(rho C) = tau_max;
    # an edge never reinforced falls to tau_min
    n, rho, C = 12, 0.1, 1000
    tmax, tmin = O.limits(n, rho, 0.01, C)
    persist = O.persist_factor(rho)
    tau = np.full((n, n), tmin, np.float32)
    tour = np.arange(n, dtype=np.int32)
    for _ in range(400):
        tau = O.evaporate(tau, persist, tmin, tmax)
        tau = O.deposit(tau, tour, np.float32(1.0 / C), tmax)
    assert abs(tau[0, 1] / tmax - 1.0) < 1e-4
    assert tau[0, 2] == tmin
    assert np.all(tau <= tmax) and np.all(tau >= tmin)


def test_colony_set_pheromone_sets_the_state():
    n = 40
    col = O.Colony(xy=I.uniform(n, 5), m=4, cl=8, alpha=1.0)
    tau = I.random_pheromone(n, 11, 1e-5, 1e-3)
    col.set_pheromone(tau, np.float32(1e-5), np.float32(1e-3))
    st = col.state()
    assert np.array_equal(st["tau"], tau)
    assert col.limits() == (np.float32(1e-5), np.float32(1e-3))
    # alpha = 1: choice_info is the single-precision product, as the pass computes it
    assert np.array_equal(st["choice"], (tau * st["eta_beta"]).astype(np.float32))
