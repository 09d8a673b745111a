"""Pins of the learned-prior oracle (oracle/prior_oracle.py) by what does not
come from the oracle itself: an independent bf16 conversion, closed forms,
symmetry, finite differences and hand-checked features."""
import numpy as np
import pytest

import oracle as O
from oracle import prior_oracle as P
from paper_2003_11902_gb300 import instances as I


def _graph(n, seed):
    xy = I.uniform(n, seed)
    d = O.distances(xy)
    nn = O.candidates(d, P.K_NN)
    return xy, d, nn


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(10000).astype(np.float32) * 10
    x[:4] = [0.0, -0.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8]  # ties to even
    want = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    assert np.array_equal(P.bf16(x), want)


def test_parameter_layout():
    assert P.N_PARAMS == 29442
    v = np.arange(P.N_PARAMS, dtype=np.float64)
    assert np.array_equal(P.pack(P.unpack(v)), v)


def test_features_by_hand():
    # a 3 x 3 lattice with spacing 10 at offset (5, 7): centre (15, 17), side 20
    xy = np.array([[5 + 10 * i, 7 + 10 * j] for j in range(3) for i in range(3)], np.int32)
    d = O.distances(xy)
    nn = np.argsort(d + np.eye(9, dtype=np.int64) * 10**9, axis=1, kind="stable")[:, :8]
    # only 8 neighbours exist; pad the list to 16 by repeating the farthest
    nn16 = np.concatenate([nn, np.repeat(nn[:, 7:8], 8, axis=1)], axis=1)
    F, dn = P.features(xy, d, nn16)
    assert F[4, 0] == 0.0 and F[4, 1] == 0.0          # the centre node
    assert F[0, 0] == -0.5 and F[8, 1] == 0.5
    D = float(d[0, nn16[0, 15]])                       # = max over nodes of the 16th distance
    assert D == 28.0                                   # corner to opposite corner, rounded sqrt(800)
    assert F[4, 2] == np.float32(10 / D) and F[4, 5] == np.float32(14 / D)
    assert np.all(F[:, 6] == 1) and np.all(F[:, 7] == 0)


def test_zero_weights_give_the_distance_term():
    xy, d, nn = _graph(60, 3)
    F, dn = P.features(xy, d, nn)
    p = P.unpack(np.zeros(P.N_PARAMS))
    p["a"][0], p["c"][0] = -2.0, 0.5
    s, _ = P.forward(P.pack(p), F, dn, nn, gpu_rounding=False)
    np.testing.assert_allclose(s, -2.0 * dn.astype(np.float64) + 0.5, rtol=0, atol=1e-12)


def test_scores_follow_a_relabelling_of_the_nodes():
    xy, d, nn = _graph(50, 4)
    params = I.prior_params(5)
    F, dn = P.features(xy, d, nn)
    s, _ = P.forward(params, F, dn, nn, gpu_rounding=False)
    perm = np.random.default_rng(1).permutation(50)      # new label of old node v is inv[v]
    inv = np.argsort(perm)
    xy2 = xy[perm]
    d2 = O.distances(xy2)
    nn2 = O.candidates(d2, P.K_NN)
    F2, dn2 = P.features(xy2, d2, nn2)
    s2, _ = P.forward(params, F2, dn2, nn2, gpu_rounding=False)
    # node perm[i] of the old labelling is node i now; compare edge by edge
    for i in range(50):
        old = {int(v): s[perm[i], k] for k, v in enumerate(nn[perm[i]])}
        for k, v in enumerate(nn2[i]):
            assert abs(s2[i, k] - old[int(perm[v])]) < 1e-9


def test_backward_matches_finite_differences():
    xy, d, nn = _graph(40, 6)
    F, dn = P.features(xy, d, nn)
    params = I.prior_params(7)
    y = P.labels(nn, I.random_permutation(40, 8))
    s, cache = P.forward(params, F, dn, nn, gpu_rounding=False)
    g = P.backward(params, cache, y)
    rng = np.random.default_rng(9)
    idx = list(rng.choice(P.N_PARAMS - 2, 40, replace=False)) + [P.N_PARAMS - 2, P.N_PARAMS - 1]
    for j in idx:
        e = np.zeros(P.N_PARAMS)
        e[j] = 1e-6
        lp = P.loss(P.forward(params + e, F, dn, nn, gpu_rounding=False)[0], y)
        lm = P.loss(P.forward(params - e, F, dn, nn, gpu_rounding=False)[0], y)
        fd = (lp - lm) / 2e-6
        assert abs(fd - g[j]) <= 1e-6 + 1e-4 * abs(fd), (j, fd, g[j])


def test_labels_mark_tour_edges_both_ways():
    xy, d, nn = _graph(80, 10)
    tour = O.nn_tour(d)[1] if hasattr(O, "nn_tour") else I.random_permutation(80, 1)
    y = P.labels(nn, tour)
    assert y.max() == 1 and y.sum(axis=1).max() <= 2
    succ = {int(a): int(b) for a, b in zip(tour, np.roll(tour, -1))}
    for i in range(80):
        for k in range(P.K_NN):
            j = int(nn[i, k])
            assert y[i, k] == (succ[i] == j or succ[j] == i)
