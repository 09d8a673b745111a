"""The learned edge prior on the GPU (tensor-core products) against the numpy
oracle: forward scores at the GPU's bf16 rounding points, gradients against the
fp64 backward, training that lowers the loss, and the replaced heuristic."""
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
