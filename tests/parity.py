"""Comparison rules between the CUDA path and the oracle (test helpers).

Node picks are driven by the same counters on both sides; they must agree
except where the oracle's key for the GPU's pick lies within NEAR_TIE of the
oracle's best key (relative), the tolerance the keys' float rounding needs.
After an allowed divergence the rest of that ant's tour follows a different
path and is not compared further.  Every input here comes from the oracle or
the seeded generators; GPU outputs are only compared against them.

The roulette wheel (Sec. 4.2.1) is compared by teacher forcing: every step of
a GPU tour is replayed by the oracle on the GPU's own prefix.  The oracle sums
the weights in double precision; the GPU sums them in single precision (lane
partial sums, a 5-level lane scan and a running offset over rounds of 128
positions), so its cumulative sums and its theta = u T each lie within
(R + 10) 2^-24 T of the exact values, R the number of rounds.  A pick may then
differ from the oracle's only when theta lies within roulette_slack() T of
the boundary between the two picks' intervals (the cumulative sum at the
lower of the two positions); the rate of such steps is reported.
"""
import math
from fractions import Fraction

import numpy as np

NEAR_TIE = 1e-6


def first_divergence(a, b):
    d = np.nonzero(a != b)[0]
    return int(d[0]) if len(d) else -1


def check_ant(ocol, it, ant, gpu_tour, gpu_len=None):
    """Compare one GPU tour with the oracle's tour of the same ant.

    Returns "exact" or "near_tie"; raises AssertionError on a real mismatch.
    """
    olen, otour, _ = ocol.construct(it, ant)
    t = first_divergence(otour, gpu_tour)
    if t < 0:
        if gpu_len is not None:
            assert int(gpu_len) == int(olen), f"ant {ant}: length {gpu_len} != oracle {olen}"
        return "exact"
    assert t > 0, f"ant {ant}: start node {gpu_tour[0]} != oracle {otour[0]}"
    vis = np.zeros(ocol.n, np.uint8)
    vis[otour[:t]] = 1
    mode, keys = ocol.step_keys(it, ant, t, int(otour[t - 1]), vis)
    g = int(gpu_tour[t])
    assert not np.isnan(keys[g]), f"ant {ant} step {t}: GPU picked {g}, not a competing node"
    best = keys[int(otour[t])]
    gap = (best - keys[g]) / abs(best) if best != 0 else abs(keys[g])
    assert gap <= NEAR_TIE, (f"ant {ant} step {t} (mode {mode}): GPU pick {g} key {keys[g]!r} vs "
                             f"oracle pick {otour[t]} key {best!r}, relative gap {gap:.3g}")
    return "near_tie"


def roulette_slack(npos):
    """Bound, as a fraction of the total T, on |theta - C(p)| for any position p
    under the GPU's single-precision summation (two sums of depth R + 10 and
    one product, with room to spare) plus the oracle's double rounding."""
    R = (npos + 127) // 128
    return (2 * R + 24) * 2.0 ** -24 + npos * 2.0 ** -50


def check_ant_variant(ocol, it, ant, gpu_tour, counts=None):
    """Teacher-forced comparison of one GPU whole-row variant tour.

    Every step t replays the oracle on gpu_tour[:t].  Roulette wheel: a
    different pick is allowed only at a near-boundary draw (see the module
    docstring); reservoir sampling over the compact list: only at a near-tie.
    Updates and returns `counts` ({"steps", "boundary", "near_tie"})."""
    from oracle import start_node
    counts = counts if counts is not None else {"steps": 0, "boundary": 0, "near_tie": 0}
    n = ocol.n
    gpu_tour = np.asarray(gpu_tour)
    assert is_permutation(gpu_tour, n), f"ant {ant}: not a permutation"
    assert gpu_tour[0] == start_node(ocol.seed, it, ant, n), f"ant {ant}: start node"
    for t in range(1, n):
        pick, order, val, u = ocol.variant_step(it, ant, gpu_tour, t)
        counts["steps"] += 1
        g = int(gpu_tour[t])
        if g == pick:
            continue
        pg = np.flatnonzero(order == g)
        assert len(pg) == 1, f"ant {ant} step {t}: GPU picked {g}, which is not selectable"
        pg, po = int(pg[0]), int(np.flatnonzero(order == pick)[0])
        if ocol.selection == 1:
            assert val[pg] > 0, f"ant {ant} step {t}: GPU picked {g} of weight 0"
            T = Fraction(math.fsum(val))
            lo = min(pg, po)
            C_lo = Fraction(math.fsum(val[:lo + 1]))
            theta = Fraction(u) * T
            gap = abs(theta - C_lo) / T
            assert gap <= roulette_slack(len(order)), (
                f"ant {ant} step {t}: GPU pick {g} (position {pg}) vs oracle {pick} (position {po}); "
                f"theta is {float(gap):.3g} T from the boundary, beyond the rounding bound "
                f"{roulette_slack(len(order)):.3g} T")
            counts["boundary"] += 1
        else:
            best, kg = val[po], val[pg]
            assert not np.isnan(kg), f"ant {ant} step {t}: GPU picked {g}, not a competing node"
            gap = (best - kg) / abs(best) if best != 0 else abs(kg)
            assert gap <= NEAR_TIE, (f"ant {ant} step {t}: GPU pick {g} key {kg!r} vs oracle pick "
                                     f"{pick} key {best!r}, relative gap {gap:.3g}")
            counts["near_tie"] += 1
    return counts


def is_permutation(t, n):
    return len(t) == n and np.array_equal(np.sort(t), np.arange(n))
