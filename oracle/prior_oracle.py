"""Learned edge prior -- test infrastructure only (tests, smoke and the bench's
CPU legs may use it; the library never does).

A plain numpy statement of the message-passing network that scores each
candidate edge, in this library's definition (the paper has no learned
component; it is an extension built around the MMAS of Alg. 1):

  graph     node i's neighbours are its 16 nearest nodes nn[i][0..15] (the
            candidate lists, ordered by (distance, id))
  features  F0[i] = ((x_i - cx)/s, (y_i - cy)/s, d(i,nn0)/D, d(i,nn1)/D,
            d(i,nn3)/D, d(i,nn15)/D, 1, 0), where (cx, cy) is the centre of the
            bounding box, s its longer side and D = max_i d(i, nn[i][15]) --
            exact integers and a maximum, so no summation order is involved
  input     h0 = relu(F0 W0^T + b0)                               (64 wide)
  layers    m_i = (1/16) sum_k h_{nn[i][k]};  z = [h | m];
            h <- relu(z W_l^T + b_l) + h,  l = 1, 2, 3                (W_l: 64 x 128)
  scores    q = h Wq^T;  s[i][k] = <q_i, h_{nn[i][k]}> / 8 + a dn[i][k] + c,
            dn[i][k] = d(i, nn[i][k]) / D
  loss      mean binary cross-entropy of sigmoid(s) against y[i][k] = 1 when the
            edge (i, nn[i][k]) is in a given (elite) tour

`forward(..., gpu_rounding=True)` rounds to bf16 exactly where the GPU stores
bf16 (every GEMM operand: F0, the weights, h, z) and accumulates what the GPU
accumulates in fp32 in the same order (the neighbour mean over k = 0..15, the
score dot over c = 0..63); GEMM products are exact (fp64) here, fp32 there.
`backward` is the fp64 gradient of the unrounded network.

Parameter vector (fp32, this order): W0 [64][8], b0 [64], W1 [64][128], b1,
W2, b2, W3, b3, Wq [64][64], a, c  -- 29,442 values.
"""
from __future__ import annotations

import numpy as np

H = 64
K_NN = 16
F_IN = 8
SHAPES = [("W0", (H, F_IN)), ("b0", (H,)), ("W1", (H, 2 * H)), ("b1", (H,)),
          ("W2", (H, 2 * H)), ("b2", (H,)), ("W3", (H, 2 * H)), ("b3", (H,)),
          ("Wq", (H, H)), ("a", (1,)), ("c", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(vec):
    vec = np.asarray(vec)
    out, o = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = vec[o:o + size].reshape(shape)
        o += size
    assert o == vec.size == N_PARAMS
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return (rounded.astype(np.uint32) << 16).view(np.float32).reshape(np.shape(x))


def features(xy, d, nn):
    """F0 [n][8] float32 and dn [n][16] float32 (see the module docstring)."""
    xy = np.asarray(xy, np.int64)
    n = xy.shape[0]
    lo, hi = xy.min(axis=0), xy.max(axis=0)
    cx, cy = (lo[0] + hi[0]) / 2.0, (lo[1] + hi[1]) / 2.0
    s = float(max(hi[0] - lo[0], hi[1] - lo[1], 1))
    dk = np.take_along_axis(np.asarray(d, np.int64), np.asarray(nn, np.int64), axis=1)  # [n][16]
    D = float(max(int(dk[:, K_NN - 1].max()), 1))
    F = np.zeros((n, F_IN), np.float32)
    F[:, 0] = ((xy[:, 0] - cx) / s).astype(np.float32)
    F[:, 1] = ((xy[:, 1] - cy) / s).astype(np.float32)
    F[:, 2] = (dk[:, 0] / D).astype(np.float32)
    F[:, 3] = (dk[:, 1] / D).astype(np.float32)
    F[:, 4] = (dk[:, 3] / D).astype(np.float32)
    F[:, 5] = (dk[:, 15] / D).astype(np.float32)
    F[:, 6] = 1.0
    dn = (dk / D).astype(np.float32)
    return F, dn


def _mean_nbr32(h, nn):
    """(1/16) sum_k h[nn[i][k]] accumulated in float32, k = 0..15 in order."""
    acc = np.zeros_like(h, dtype=np.float32)
    for k in range(K_NN):
        acc = (acc + h[nn[:, k]]).astype(np.float32)
    return (acc * np.float32(1.0 / K_NN)).astype(np.float32)


def _rounding(gpu_rounding):
    return bf16 if gpu_rounding else (lambda x: np.asarray(x, np.float64))


def _lin(x, W, b, r):
    """x W^T (+ b): the exact product (fp64) of the operands after rounding r."""
    y = r(x).astype(np.float64) @ r(W).astype(np.float64).T
    if b is not None:
        y = y + np.asarray(b, np.float64)
    return y


def input_layer(F, W0, b0, gpu_rounding):
    """h0 = relu(F0 W0^T + b0): fp32 after bf16 operands, else fp64."""
    f = np.float32 if gpu_rounding else np.float64
    return np.maximum(_lin(F, W0, b0, _rounding(gpu_rounding)), 0.0).astype(f)


def mp_layer(h, nn, W, b, gpu_rounding):
    """One message-passing layer: m_i = mean_k h[nn[i][k]], z = [h | m],
    h' = relu(z W^T + b) + h.  Rounded: the mean of the bf16 h summed in fp32
    over k = 0..15 in order, z in bf16, h' stored in fp32.  Returns (h', z, pre)."""
    r = _rounding(gpu_rounding)
    if gpu_rounding:
        m = _mean_nbr32(r(h), nn)
    else:
        m = np.asarray(h, np.float64)[nn].mean(axis=1)
    z = np.concatenate([r(h), r(m)], axis=1)
    pre = _lin(z, W, b, r)
    f = np.float32 if gpu_rounding else np.float64
    return (np.maximum(pre, 0.0) + h).astype(f), z, pre


def query(h, Wq, gpu_rounding):
    """q = h Wq^T (fp32 after bf16 operands, else fp64)."""
    f = np.float32 if gpu_rounding else np.float64
    return _lin(h, Wq, None, _rounding(gpu_rounding)).astype(f)


def edge_scores(q, h, nn, dn, a, c, gpu_rounding):
    """s[i][k] = <q_i, h[nn[i][k]]> / 8 + a dn[i][k] + c.  Rounded: h in bf16,
    the dot summed in fp32 over c = 0..63 in order, a and c in fp32."""
    if gpu_rounding:
        hb = bf16(h)
        dot = np.zeros(nn.shape, np.float32)
        for ch in range(H):  # float32, c = 0..63 in order
            dot = (dot + q[:, ch][:, None] * hb[nn, ch]).astype(np.float32)
        return (dot * np.float32(0.125) + np.float32(a) * dn + np.float32(c)).astype(np.float32)
    q = np.asarray(q, np.float64)
    h = np.asarray(h, np.float64)
    return np.einsum("ic,ikc->ik", q, h[nn]) / 8.0 + a * np.asarray(dn, np.float64) + c


def forward(params, F, dn, nn, gpu_rounding=True):
    """Scores s [n][16] (float32 when gpu_rounding, else float64) and the cache.
    The same stages in both modes; only their rounding differs."""
    p = unpack(params)
    nn = np.asarray(nn, np.int64)
    cache = {"F": F, "dn": dn, "nn": nn}
    h = input_layer(F, p["W0"], p["b0"], gpu_rounding)
    cache["h0"] = h
    for l in (1, 2, 3):
        h, z, pre = mp_layer(h, nn, p[f"W{l}"], p[f"b{l}"], gpu_rounding)
        cache[f"z{l}"], cache[f"pre{l}"], cache[f"h{l}"] = z, pre, h
    q = query(h, p["Wq"], gpu_rounding)
    cache["q"] = q
    s = edge_scores(q, h, nn, dn, p["a"][0], p["c"][0], gpu_rounding)
    return s, cache


def loss(s, y):
    """Mean binary cross-entropy with logits, in float64."""
    s = np.asarray(s, np.float64)
    return float(np.mean(np.maximum(s, 0) - s * y + np.log1p(np.exp(-np.abs(s)))))


def backward(params, cache, y):
    """Gradient of loss(forward(params, gpu_rounding=False)) in float64."""
    p = {k: np.asarray(v, np.float64) for k, v in unpack(params).items()}
    nn, dn = cache["nn"], np.asarray(cache["dn"], np.float64)
    n = nn.shape[0]
    s, c2 = forward(params, cache["F"], cache["dn"], nn, gpu_rounding=False)
    g = {k: np.zeros_like(v) for k, v in p.items()}
    ds = (1.0 / (1.0 + np.exp(-s)) - y) / s.size
    h = c2["h3"]
    q = c2["q"]
    g["a"][0] = np.sum(ds * dn)
    g["c"][0] = np.sum(ds)
    dq = np.einsum("ik,ikc->ic", ds, h[nn]) / 8.0
    dh = np.zeros_like(h)
    np.add.at(dh, nn.ravel(), (ds[:, :, None] * q[:, None, :]).reshape(-1, H) / 8.0)
    g["Wq"] = dq.T @ h
    dh += dq @ p["Wq"]
    for l in (3, 2, 1):
        pre, z = c2[f"pre{l}"], c2[f"z{l}"]
        da = dh * (pre > 0)
        g[f"W{l}"] = da.T @ z
        g[f"b{l}"] = da.sum(axis=0)
        dz = da @ p[f"W{l}"]
        dh_in = dh + dz[:, :H]
        dm = dz[:, H:] / K_NN
        np.add.at(dh_in, nn.ravel(), np.repeat(dm, K_NN, axis=0))
        dh = dh_in
    pre0 = np.asarray(cache["F"], np.float64) @ p["W0"].T + p["b0"]
    da0 = dh * (pre0 > 0)
    g["W0"] = da0.T @ np.asarray(cache["F"], np.float64)
    g["b0"] = da0.sum(axis=0)
    return pack(g)


# Adam's hyperparameters as the library holds them: single-precision values
ADAM_B1, ADAM_B2, ADAM_EPS = float(np.float32(0.9)), float(np.float32(0.999)), float(np.float32(1e-8))


def adam_step(theta, g, m, v, t, lr, b1=ADAM_B1, b2=ADAM_B2, eps=ADAM_EPS):
    """Step t (t >= 1) of Adam (Kingma and Ba, ICLR 2015, Algorithm 1) in
    float64: m <- b1 m + (1 - b1) g; v <- b2 v + (1 - b2) g^2;
    m_hat = m / (1 - b1^t); v_hat = v / (1 - b2^t);
    theta <- theta - lr m_hat / (sqrt(v_hat) + eps).  Returns (theta, m, v)."""
    g = np.asarray(g, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * g * g
    m_hat = m / (1.0 - b1 ** t)
    v_hat = v / (1.0 - b2 ** t)
    return np.asarray(theta, np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def labels(nn, tour):
    """y[i][k] = 1 when (i, nn[i][k]) is an edge of the closed tour."""
    tour = np.asarray(tour)
    n = tour.size
    succ = np.empty(n, np.int64)
    pred = np.empty(n, np.int64)
    succ[tour] = np.roll(tour, -1)
    pred[tour] = np.roll(tour, 1)
    nn = np.asarray(nn)
    return ((nn == succ[:, None]) | (nn == pred[:, None])).astype(np.float64)
