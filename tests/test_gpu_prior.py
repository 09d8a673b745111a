"""The learned edge prior on the GPU (tensor-core products) against the numpy
oracle: forward scores at the GPU's bf16 rounding points (up to n = 18,500),
gradients against the fp64 backward element by element, Adam steps against
Kingma and Ba's rule, training that lowers the loss, and the replaced or
weighted heuristic entry by entry."""
import numpy as np
import pytest

import oracle as O
from oracle import prior_oracle as P
from paper_2003_11902_gb300 import Colony, MMASError, Prior, instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _setup(n, seed, cl=16):
    xy = I.uniform(n, seed)
    col = Colony(xy=xy, m=8, cl=cl, seed=1)
    s = col.setup()
    nn = s["cand"][:, :16].astype(np.int64)
    F, dn = P.features(xy, s["d"], nn)
    return xy, col, s, nn, F, dn


@pytest.mark.parametrize("n,cl,seed", [(37, 16, 3), (300, 16, 4), (2000, 32, 5)])
def test_scores_match_the_oracle(n, cl, seed):
    xy, col, s, nn, F, dn = _setup(n, 700 + n, cl)
    params = I.prior_params(seed)
    pr = Prior(params)
    got = pr.scores(col)
    want, _ = P.forward(params, F, dn, nn, gpu_rounding=True)
    err = np.abs(got - want)
    # fp32 accumulation order inside the products can flip a bf16 rounding of
    # an activation; such flips are rare and one bf16 ulp (2^-8 relative) each
    assert np.quantile(err, 0.99) <= 1e-3 * (1 + np.abs(want).max())
    assert err.max() <= 3e-2 * (1 + np.abs(want).max())
    pr.close()
    col.close()


def test_gradient_matches_the_oracle():
    xy, col, s, nn, F, dn = _setup(400, 31)
    params = I.prior_params(8)
    tour = O.nn_tour(s["d"])[1]
    pr = Prior(params)
    g, loss = pr.grad(col, tour)
    y = P.labels(nn, tour)
    s0, cache = P.forward(params, F, dn, nn, gpu_rounding=False)
    want = P.backward(params, cache, y)
    assert abs(loss - P.loss(s0, y)) <= 2e-3 * abs(P.loss(s0, y))
    cos = float(g @ want / (np.linalg.norm(g) * np.linalg.norm(want)))
    assert cos > 0.995, cos
    assert np.linalg.norm(g - want) <= 0.06 * np.linalg.norm(want)
    assert np.array_equal(pr.params(), params)  # the gradient pass leaves the parameters alone
    pr.close()
    col.close()


@pytest.mark.parametrize("n,seed", [(400, 31), (2000, 33)])
def test_gradient_matches_the_oracle_element_by_element(n, seed):
    # Every element of every parameter block (W0 .. Wq, every bias, a and c)
    # against the fp64 gradient of the unrounded network.  The GPU rounds
    # operands to bf16 (unit roundoff 2^-8) at about ten stages on the way to
    # a gradient element (four forward products, the score head, four
    # backward products, the final weight-gradient product), so a first-order
    # estimate puts each element within 10 * 2^-8 of the size of its terms;
    # |g| plus the block's RMS stands for that size, since terms can cancel.
    # (Observed: at most 0.03, 99th percentile 0.013, median 5e-4.)
    xy, col, s, nn, F, dn = _setup(n, seed)
    params = I.prior_params(8)
    tour = O.nn_tour(s["d"])[1]
    pr = Prior(params)
    g, _ = pr.grad(col, tour)
    y = P.labels(nn, tour)
    _, cache = P.forward(params, F, dn, nn, gpu_rounding=False)
    want = P.unpack(P.backward(params, cache, y))
    got = P.unpack(g.astype(np.float64))
    tol = 10 * 2.0 ** -8
    for name, w in want.items():
        w = w.ravel()
        rms = np.sqrt(np.mean(w * w))
        rel = np.abs(got[name].ravel() - w) / (np.abs(w) + rms)
        assert rel.max() <= tol, f"{name}: worst {rel.max():.4f} at element {int(rel.argmax())}"
        print(f"{name}: worst {rel.max():.4f}, median {np.median(rel):.2e}")
    pr.close()
    col.close()


def test_training_lowers_the_loss_and_apply_replaces_the_heuristic():
    xy = I.uniform(500, 77)
    col = Colony(xy=xy, m=500, cl=16, seed=2)
    col.iterate(30)
    _, elite = col.best_tour()
    pr = Prior(I.prior_params(9))
    first = pr.train(col, elite, steps=1, lr=3e-3)
    last = pr.train(col, elite, steps=60, lr=3e-3)
    assert last < 0.8 * first, (first, last)
    scores = pr.scores(col)
    pr.apply(col)
    st = col.setup()
    eb = st["eta_beta"]
    nn = st["cand"][:, :16]
    rows = np.arange(500)[:, None]
    np.testing.assert_allclose(eb[rows, nn], 1 / (1 + np.exp(-scores.astype(np.float64))), rtol=1e-5)
    col.iterate(3)
    tours, lens = col.tours()
    assert all(sorted(t) == list(range(500)) for t in tours)
    assert col.best_tour()[0] > 0
    pr.close()
    col.close()


def test_prior_needs_coordinates_and_16_candidates():
    pr = Prior()
    col = Colony(xy=I.uniform(60, 1), m=4, cl=8)
    with pytest.raises(MMASError, match="length >= 16"):
        pr.scores(col)
    col.close()
    col = Colony(dist=O.distances(I.uniform(60, 1)), m=4, cl=16)
    with pytest.raises(MMASError, match="coordinates"):
        pr.apply(col)
    col.close()
    pr.close()


def test_weighted_apply_scales_the_heuristic():
    xy = I.uniform(300, 91)
    col = Colony(xy=xy, m=8, cl=16, seed=2)
    eb0 = col.setup()["eta_beta"].astype(np.float64)
    pr = Prior(I.prior_params(4))
    pr.apply_weighted(col, 0.0)  # gamma = 0: plain MMAS
    assert np.array_equal(col.setup()["eta_beta"], eb0.astype(np.float32))
    s = pr.scores(col).astype(np.float64)
    p = 1 / (1 + np.exp(-s))
    pr.apply_weighted(col, 2.0)
    st = col.setup()
    eb, nn = st["eta_beta"].astype(np.float64), st["cand"][:, :16]
    rows = np.arange(300)[:, None]
    np.testing.assert_allclose(eb[rows, nn], eb0[rows, nn] * p ** 2, rtol=1e-5)
    mask = np.ones_like(eb, bool)
    mask[rows, nn] = False
    scale = (p.min(axis=1) ** 2)[:, None] * np.ones_like(eb)
    np.testing.assert_allclose(eb[mask], (eb0 * scale)[mask], rtol=1e-5)
    col.iterate(2)
    tours, _ = col.tours()
    assert all(sorted(t) == list(range(300)) for t in tours)
    with pytest.raises(MMASError, match="gamma"):
        pr.apply_weighted(col, -1.0)
    pr.close()
    col.close()


def test_adam_steps_match_the_oracle():
    # three training steps; each is checked against Adam (Kingma and Ba) in
    # float64 applied to the gradient that step used, element by element:
    # m and v within a few float roundings of their two terms, theta within
    # one ulp of itself plus a few roundings of the step
    xy, col, s, nn, F, dn = _setup(300, 41)
    params = I.prior_params(12)
    pr = Prior(params)
    tour = I.random_permutation(300, 5)
    lr = float(np.float32(2e-3))  # the library takes lr as a float
    theta = params.astype(np.float64)
    m0, v0, _, t0 = pr.state()
    assert t0 == 0 and not m0.any() and not v0.any()
    m, v = m0.astype(np.float64), v0.astype(np.float64)
    u = 2.0 ** -24
    for t in range(1, 4):
        pr.train(col, tour, steps=1, lr=lr)
        gm, gv, g, step = pr.state()
        assert step == t
        gp = pr.params().astype(np.float64)
        want_th, want_m, want_v = P.adam_step(theta, g, m, v, t, lr)
        g64 = g.astype(np.float64)
        tol_m = 4 * u * (P.ADAM_B1 * np.abs(m) + (1 - P.ADAM_B1) * np.abs(g64)) + 1e-38
        tol_v = 6 * u * (P.ADAM_B2 * v + (1 - P.ADAM_B2) * g64 * g64) + 1e-38
        assert np.all(np.abs(gm - want_m) <= tol_m), np.max(np.abs(gm - want_m) / tol_m)
        assert np.all(np.abs(gv - want_v) <= tol_v), np.max(np.abs(gv - want_v) / tol_v)
        step_sz = np.abs(want_th - theta)
        tol_p = np.spacing(np.abs(want_th).astype(np.float32)).astype(np.float64) + 16 * u * step_sz
        assert np.all(np.abs(gp - want_th) <= tol_p), np.max(np.abs(gp - want_th) / tol_p)
        theta, m, v = gp, gm.astype(np.float64), gv.astype(np.float64)
    pr.close()
    col.close()


def test_optimiser_state_round_trips():
    xy, col, s, nn, F, dn = _setup(120, 43)
    pr = Prior(I.prior_params(2))
    tour = I.random_permutation(120, 2)
    pr.train(col, tour, steps=2, lr=1e-3)
    m, v, g, t = pr.state()
    p2 = pr.params()
    pr.train(col, tour, steps=1, lr=1e-3)
    after = pr.params()
    # restore parameters (which resets the moments) and then the moments: the
    # next step repeats
    pr.set_params(p2)
    assert pr.state()[3] == 0
    pr.set_state(m, v, t)
    pr.train(col, tour, steps=1, lr=1e-3)
    np.testing.assert_allclose(pr.params(), after, rtol=0, atol=1e-6)
    with pytest.raises(MMASError, match="v finite"):
        pr.set_state(m, -np.ones_like(v), 1)
    pr.close()
    col.close()


def test_apply_scales_every_other_entry_of_the_row():
    # replace mode: candidates take sigmoid(s); every other entry j of row i is
    # d_ij^-beta times min_k sigmoid(s_ik) / (the 16th candidate's d^-beta)
    xy = I.uniform(300, 93)
    col = Colony(xy=xy, m=8, cl=16, seed=2)
    st0 = col.setup()
    eb0 = st0["eta_beta"].astype(np.float64)
    nn = st0["cand"][:, :16]
    pr = Prior(I.prior_params(6))
    p = 1 / (1 + np.exp(-pr.scores(col).astype(np.float64)))
    pr.apply(col)
    eb = col.setup()["eta_beta"].astype(np.float64)
    rows = np.arange(300)[:, None]
    scale = p.min(axis=1) / eb0[np.arange(300), nn[:, 15]]
    want = eb0 * scale[:, None]
    want[rows, nn] = p
    mask = np.ones_like(eb, bool)
    mask[rows, nn] = False
    np.fill_diagonal(mask, False)
    np.testing.assert_allclose(eb[mask], want[mask], rtol=1e-5)
    np.testing.assert_allclose(eb[rows, nn], p, rtol=1e-5)
    assert np.all(np.diag(eb) == 0)
    # every non-candidate entry stays at most the row's smallest candidate value
    assert np.all(eb[mask].reshape(-1) <= np.repeat(p.min(axis=1), 300 - 17) * (1 + 1e-6))
    pr.close()
    col.close()


def test_scores_match_the_oracle_at_n18500():
    # the size of the largest learned-prior workload (uniform, 18,500 nodes)
    n = 18500
    xy = I.uniform(n, 1018)
    col = Colony(xy=xy, m=8, cl=16, seed=1)
    s = col.setup()
    nn = s["cand"].astype(np.int64)
    F, dn = P.features(xy, s["d"], nn)
    del s
    params = I.prior_params(3)
    pr = Prior(params)
    got = pr.scores(col)
    want, _ = P.forward(params, F, dn, nn, gpu_rounding=True)
    err = np.abs(got - want)
    assert np.quantile(err, 0.99) <= 1e-3 * (1 + np.abs(want).max())
    assert err.max() <= 3e-2 * (1 + np.abs(want).max())
    print(f"n = 18500: 99th percentile {np.quantile(err, 0.99):.3g}, max {err.max():.3g}, "
          f"exact {np.mean(err == 0):.3f}")
    pr.close()
    col.close()
