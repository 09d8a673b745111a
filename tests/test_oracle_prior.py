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


# ---------------------------------------------------------------------------
# The forward pass at the GPU's rounding points, pinned to the unrounded one.
#
# forward() chains four stages (input layer, three message-passing layers, the
# query, the edge scores), the same in both modes.  Each stage is checked on its
# own: fed the SAME input (the rounded pass's own activations), its rounded form
# (bf16 GEMM operands, unit roundoff 2^-8; fp32 storage and fp32 sums, unit
# roundoff 2^-24) must lie element by element within a bound on that stage's
# rounding alone from its unrounded form.  For a product with rounded operands,
# A'B' - AB = (A' - A)B' + A(B' - B), so |A'B' - AB| <= |A' - A||B'| + |A||B' - B|;
# relu and the residual add are 1-Lipschitz; an fp32 sum of k terms is off by at
# most k 2^-24 times the sum of their magnitudes, and each fp32 store by 2^-24 of
# the value stored.  A mistake confined to the rounded path (a swapped half of z,
# a dropped term, a wrong neighbour) moves a stage by O(1) and breaks its bound.

UF = 2.0 ** -24
SLACK = 1 + 1e-6


def _b64(x):
    return P.bf16(np.asarray(x, np.float32)).astype(np.float64)


def _abs_err_of_product(x, W):
    """|bf16(x) bf16(W)^T - x W^T| bound, element by element."""
    x = np.asarray(x, np.float64)
    W = np.asarray(W, np.float64)
    return np.abs(_b64(x) - x) @ np.abs(_b64(W)).T + np.abs(x) @ np.abs(_b64(W) - W).T


def _mp_bound(x, nn, W, hr):
    """Bound on |rounded - unrounded| of one message-passing layer on input x."""
    x64 = np.asarray(x, np.float64)
    xb = _b64(x)
    m32 = P._mean_nbr32(P.bf16(x), nn).astype(np.float64)     # the fp32 mean of bf16 h
    m_exact = x64[nn].mean(axis=1)
    # |m32 - m| <= mean |bf16(h) - h| + the fp32 sum's rounding
    Em = np.abs(xb - x64)[nn].mean(axis=1) + P.K_NN * UF * np.abs(xb[nn]).mean(axis=1)
    Ez = np.concatenate([np.abs(xb - x64), np.abs(_b64(m32) - m32) + Em], axis=1)
    W = np.asarray(W, np.float64)
    Epre = Ez @ np.abs(_b64(W)).T + np.abs(np.concatenate([x64, m_exact], axis=1)) @ np.abs(_b64(W) - W).T
    return (Epre + UF * np.abs(hr)) * SLACK


def _check_stages(params, F, dn, nn):
    p = P.unpack(np.asarray(params, np.float64))
    nn = np.asarray(nn, np.int64)
    _, cr = P.forward(params, F, dn, nn, gpu_rounding=True)
    worst = []
    # input layer on F
    hr = P.input_layer(F, p["W0"], p["b0"], True)
    he = P.input_layer(F, p["W0"], p["b0"], False)
    bound = (_abs_err_of_product(F, p["W0"]) + UF * np.abs(hr)) * SLACK
    worst.append(np.max(np.abs(hr - he) / bound))
    assert np.array_equal(hr, cr["h0"])
    # message-passing layers, each on the rounded pass's own input
    for l in (1, 2, 3):
        x = cr[f"h{l - 1}"]
        hr, zr, _ = P.mp_layer(x, nn, p[f"W{l}"], p[f"b{l}"], True)
        he, ze, _ = P.mp_layer(x, nn, p[f"W{l}"], p[f"b{l}"], False)
        assert np.array_equal(hr, cr[f"h{l}"])
        worst.append(np.max(np.abs(hr - he) / _mp_bound(x, nn, p[f"W{l}"], hr)))
        assert np.array_equal(zr[:, :P.H], P.bf16(x))              # z = [h | m] in that order
    # query on h3
    x = cr["h3"]
    qr = P.query(x, p["Wq"], True)
    qe = P.query(x, p["Wq"], False)
    assert np.array_equal(qr, cr["q"])
    bound = (_abs_err_of_product(x, p["Wq"]) + UF * np.abs(qr)) * SLACK
    worst.append(np.max(np.abs(qr - qe) / bound))
    # edge scores on (q, h3): bf16 h, fp32 products and sums (two roundings a
    # term), fp32 a and c and three fp32 operations at the end
    a, c = p["a"][0], p["c"][0]
    sr = P.edge_scores(qr, x, nn, dn, a, c, True)
    se = P.edge_scores(qr, x, nn, dn, a, c, False)
    q64 = np.asarray(qr, np.float64)
    x64 = np.asarray(x, np.float64)
    xb = _b64(x)
    dn64 = np.asarray(dn, np.float64)
    a32, c32 = float(np.float32(a)), float(np.float32(c))
    Edot = (np.einsum("ic,ikc->ik", np.abs(q64), np.abs(xb - x64)[nn])
            + 2 * P.H * UF * np.einsum("ic,ikc->ik", np.abs(q64), np.abs(xb[nn])))
    dot = np.einsum("ic,ikc->ik", q64, xb[nn])
    bound = (Edot / 8 + abs(a - a32) * dn64 + abs(c - c32)
             + 4 * UF * (np.abs(dot) / 8 + abs(a32) * dn64 + abs(c32))) * SLACK + 1e-30
    worst.append(np.max(np.abs(sr.astype(np.float64) - se) / bound))
    return worst


def _prior_case(n, seed):
    xy, d, nn = _graph(n, seed)
    F, dn = P.features(xy, d, nn)
    params = I.prior_params(seed).astype(np.float64)
    rng = np.random.default_rng(seed)
    q = P.unpack(params)
    for name in ("b0", "b1", "b2", "b3"):
        q[name][:] = rng.normal(0, 0.2, q[name].shape)
    q["c"][0] = 0.3
    return P.pack(q).astype(np.float32).astype(np.float64), F, dn, nn


@pytest.mark.parametrize("n,seed", [(60, 21), (400, 22)])
def test_rounded_forward_stages_within_their_rounding_bounds(n, seed):
    params, F, dn, nn = _prior_case(n, seed)
    worst = _check_stages(params, F, dn, nn)
    print("worst error / bound per stage:", [f"{w:.3f}" for w in worst])
    assert all(w <= 1.0 for w in worst)
    assert all(w > 0 for w in worst)  # every stage really rounds


def test_rounded_stage_bound_catches_a_swapped_message():
    # a planted mistake in the rounded pass only: the layer computed with z =
    # [m | h] (equivalently, the halves of W_l exchanged) leaves the stage's
    # bound for a good share of the elements (the rest sit where relu cuts the
    # layer off in both), while the correct rounded layer stays inside it
    params, F, dn, nn = _prior_case(200, 23)
    nn = np.asarray(nn, np.int64)
    p = P.unpack(params)
    _, cr = P.forward(params, F, dn, nn, gpu_rounding=True)
    x = cr["h1"]
    W = p["W2"]
    Wswap = np.concatenate([W[:, P.H:], W[:, :P.H]], axis=1)
    he, _, _ = P.mp_layer(x, nn, W, p["b2"], False)
    good, _, _ = P.mp_layer(x, nn, W, p["b2"], True)
    bad, _, _ = P.mp_layer(x, nn, Wswap, p["b2"], True)
    assert np.all(np.abs(good - he) <= _mp_bound(x, nn, W, good))
    ratio = np.abs(bad - he) / _mp_bound(x, nn, W, bad)
    assert np.mean(ratio > 1) > 0.2 and ratio.max() > 10


def test_whole_rounded_forward_stays_near_the_unrounded_one():
    # end to end, the rounding of four stages moves each score by well under
    # one percent of the score range (observed on this case: ~0.3%)
    params, F, dn, nn = _prior_case(400, 24)
    sr, _ = P.forward(params, F, dn, nn, gpu_rounding=True)
    se, _ = P.forward(params, F, dn, nn, gpu_rounding=False)
    assert np.max(np.abs(sr - se)) < 1e-2 * (np.abs(se).max() + 1)


# ---------------------------------------------------------------------------
# Adam (Kingma and Ba, Algorithm 1)

def test_adam_constant_gradient_closed_form():
    # with m = v = 0 and a constant gradient g the bias corrections make
    # m_hat = g and v_hat = g^2 at every step, so each step moves theta by
    # lr g / (|g| + eps): t steps move it by t lr g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3, -2e-9, 0.0])
    theta = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    m = np.zeros(5)
    v = np.zeros(5)
    lr = 0.01
    th = theta.copy()
    for t in range(1, 8):
        th, m, v = P.adam_step(th, g, m, v, t, lr)
    want = theta - 7 * lr * g / (np.abs(g) + P.ADAM_EPS)
    np.testing.assert_allclose(th, want, rtol=0, atol=1e-12)


def test_adam_moments_decay_after_one_gradient():
    # one gradient g, then zeros: m_t = b1^(t-1) (1 - b1) g and
    # v_t = b2^(t-1) (1 - b2) g^2
    g = np.array([0.7, -1.3])
    th, m, v = P.adam_step(np.zeros(2), g, np.zeros(2), np.zeros(2), 1, 0.1)
    for t in range(2, 6):
        th, m, v = P.adam_step(th, np.zeros(2), m, v, t, 0.1)
    np.testing.assert_allclose(m, P.ADAM_B1 ** 4 * (1 - P.ADAM_B1) * g, rtol=1e-13)
    np.testing.assert_allclose(v, P.ADAM_B2 ** 4 * (1 - P.ADAM_B2) * g * g, rtol=1e-13)


def test_adam_matches_torch_optimizer():
    # torch.optim.Adam implements the same algorithm; run both on the same
    # gradient sequence in float64
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    theta0 = rng.standard_normal(50)
    grads = rng.standard_normal((6, 50)) * rng.uniform(1e-4, 10, 50)
    w = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([w], lr=0.05, betas=(P.ADAM_B1, P.ADAM_B2), eps=P.ADAM_EPS)
    th, m, v = theta0.copy(), np.zeros(50), np.zeros(50)
    for t, g in enumerate(grads, start=1):
        w.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        th, m, v = P.adam_step(th, g, m, v, t, 0.05)
    np.testing.assert_allclose(th, w.detach().numpy(), rtol=1e-12, atol=1e-14)
