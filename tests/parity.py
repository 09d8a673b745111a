"""Comparison rules between the CUDA path and the oracle (test helpers).

Node picks are driven by the same counters on both sides; they must agree
except where the oracle's key for the GPU's pick lies within NEAR_TIE of the
oracle's best key (relative), the tolerance the keys' float rounding needs.
After an allowed divergence the rest of that ant's tour follows a different
path and is not compared further.  Every input here comes from the oracle or
the seeded generators; GPU outputs are only compared against them.
"""
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


def is_permutation(t, n):
    return len(t) == n and np.array_equal(np.sort(t), np.arange(n))
