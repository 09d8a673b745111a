"""Pins for the oracle's node selection: Eq. (1) sampled by weighted reservoir
sampling with the logarithmic key (Alg. 3, Alg. 4, Sec. 4.2.2).

Efraimidis and Spirakis show that the largest key u^(1/w) falls on item i with
probability w_i / sum(w); the log form keeps the order. Pick frequencies are
tested against those exact probabilities by chi-square. The same test run on
the sequential roulette wheel validates the test itself.
"""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2003_11902_gb300 import instances as I

W = np.array([0.5, 3.0, 1.0, 0.25, 2.0, 1.25])


def _chi2_p(counts, probs):
    exp = probs * counts.sum()
    return stats.chisquare(counts, exp).pvalue


def test_rwm_frequencies_match_weights():
    rng = np.random.Generator(np.random.PCG64(11))
    counts = np.zeros(len(W))
    for u in rng.random(40000):
        counts[O.rwm_pick(W, u)] += 1
    assert _chi2_p(counts, W / W.sum()) > 1e-3


def test_wrs_frequencies_match_weights():
    rng = np.random.Generator(np.random.PCG64(12))
    ids = np.arange(len(W), dtype=np.int32)
    counts = np.zeros(len(W))
    for _ in range(40000):
        r = rng.random(len(W))
        r = np.where(r == 0.0, 0.5, r)
        counts[O.wrs_pick(ids, W, r)] += 1
    assert _chi2_p(counts, W / W.sum()) > 1e-3


def test_wrs_detects_a_wrong_rule():
    # the statistical test has power: the unweighted key would be rejected
    rng = np.random.Generator(np.random.PCG64(13))
    ids = np.arange(len(W), dtype=np.int32)
    counts = np.zeros(len(W))
    for _ in range(20000):
        r = rng.random(len(W))
        counts[O.wrs_pick(ids, np.ones(len(W)), r)] += 1
    assert _chi2_p(counts, W / W.sum()) < 1e-6


def test_wrs_ties_go_to_lower_id():
    ids = np.array([7, 3, 5], dtype=np.int32)
    assert O.wrs_pick(ids, np.ones(3), np.full(3, 0.5)) == 1   # id 3
    assert O.wrs_pick(ids, np.array([1.0, 1.0, 2.0]), np.array([0.25, 0.25, 0.5])) == 2
    # a zero weight gives key -inf: it only wins when nothing else competes
    assert O.wrs_pick(ids[:1], np.zeros(1), np.full(1, 0.5)) == 0
    assert O.wrs_pick(ids, np.array([0.0, 1e-30, 0.0]), np.full(3, 0.5)) == 1


def _first_two_steps(col, iters, ants):
    """(start, first pick, second pick) of every sampled ant, pheromone fixed."""
    out = []
    for it in range(iters):
        for a in range(ants):
            _, tour, _ = col.construct(it, a)
            out.append((int(tour[0]), int(tour[1]), int(tour[2])))
    return out


@pytest.mark.parametrize("cl", [0, 4])
def test_colony_steps_follow_eq1(cl):
    # a fixed pheromone field; counters vary with the iteration index
    xy = I.uniform(7, 21, side=100)
    col = O.Colony(xy=xy, m=1, cl=cl, seed=77)
    ch = col.state()["choice"].astype(np.float64)
    cand = col.state()["cand"]
    samples = _first_two_steps(col, 1500, 12)
    n = 7
    tested = 0
    for s in range(n):
        allowed = [j for j in range(n) if j != s] if cl == 0 else list(cand[s])
        picks = [p for (st, p, _) in samples if st == s]
        if len(picks) < 300:
            continue
        counts = np.array([picks.count(j) for j in allowed], float)
        probs = ch[s, allowed] / ch[s, allowed].sum()
        assert counts.sum() == len(picks)  # nothing outside the allowed set
        assert _chi2_p(counts, probs) > 1e-4
        tested += 1
    assert tested >= 5
    # second step, conditioned on (start, first pick): visited nodes drop out
    pairs = {}
    for (s, j1, j2) in samples:
        pairs.setdefault((s, j1), []).append(j2)
    for (s, j1), picks in pairs.items():
        if len(picks) < 400:
            continue
        if cl == 0:
            allowed = [j for j in range(n) if j not in (s, j1)]
        else:
            allowed = [j for j in cand[j1] if j not in (s, j1)]
            if not allowed:
                continue
        counts = np.array([picks.count(j) for j in allowed], float)
        assert counts.sum() == len(picks)
        probs = ch[j1, allowed] / ch[j1, allowed].sum()
        assert _chi2_p(counts, probs) > 1e-4


def test_greedy_fallback_takes_the_best_unvisited_choice():
    xy = I.uniform(30, 31)
    col = O.Colony(xy=xy, m=1, cl=2, seed=5, fallback=0)
    ch = col.state()["choice"]
    cand = col.state()["cand"]
    _, tour, fb = col.construct(0, 0)
    assert fb > 0
    vis = np.zeros(30, bool)
    vis[tour[0]] = True
    seen_fallback = 0
    for t in range(1, 30):
        cur = tour[t - 1]
        if all(vis[v] for v in cand[cur]):
            un = np.nonzero(~vis)[0]
            best = un[np.argmax(ch[cur, un])]  # argmax returns the first (lowest id) maximum
            assert tour[t] == best
            seen_fallback += 1
        else:
            assert tour[t] in cand[cur] and not vis[tour[t]]
        vis[tour[t]] = True
    assert seen_fallback == fb


def test_step_keys_modes():
    xy = I.uniform(12, 41)
    col = O.Colony(xy=xy, m=1, cl=3, seed=3, fallback=1)
    cand = col.state()["cand"]
    vis = np.zeros(12, np.uint8)
    vis[0] = 1
    mode, keys = col.step_keys(0, 0, 1, 0, vis)
    assert mode == 0
    assert set(np.nonzero(~np.isnan(keys))[0]) == set(cand[0])
    assert np.all(keys[~np.isnan(keys)] < 0)
    vis[cand[0]] = 1
    mode, keys = col.step_keys(0, 0, 1, 0, vis)
    assert mode == 1  # full-row reservoir over the unvisited nodes
    assert set(np.nonzero(~np.isnan(keys))[0]) == set(np.nonzero(vis == 0)[0])
