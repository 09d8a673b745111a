"""The tensor-core BF16 GEMM (tcgen05, FP32 accumulation) against the exact
product of the same bf16-rounded inputs, at shapes spanning one tile, ragged
M and K, both column tiles (64, 128) and long reductions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2003_11902_gb300 import mmas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _bf16(x):
    return torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16)


@pytest.mark.parametrize("m,n,k,relu,bias", [
    (128, 64, 64, False, False),      # exactly one tile, one K block
    (300, 64, 200, False, True),      # ragged M and K, bias
    (1000, 128, 128, True, True),     # 128-column tile, ReLU
    (7, 64, 5, False, False),         # tiny, K below one MMA
    (129, 128, 1000, False, False),   # long reduction, one row past a tile
    (2000, 37, 64, True, False),      # n not a multiple of 16 (columns guarded)
])
def test_gemm_matches_exact_product(m, n, k, relu, bias):
    rng = np.random.default_rng(m * 7 + n + k)
    a = rng.standard_normal((m, k)).astype(np.float32)
    b = rng.standard_normal((n, k)).astype(np.float32)
    ta, tb = _bf16(a).cuda(), _bf16(b).cuda()
    tbias = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda() if bias else None
    out = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
    mmas.mmas_gemm_bf16(ta.data_ptr(), k, tb.data_ptr(), k, tbias.data_ptr() if bias else None,
                        out.data_ptr(), n, m, n, k, relu)
    # exact product of the bf16-rounded operands (float64), then bias / ReLU
    want = ta.float().cpu().numpy().astype(np.float64) @ tb.float().cpu().numpy().astype(np.float64).T
    if bias:
        want += tbias.cpu().numpy()
    if relu:
        want = np.maximum(want, 0.0)
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    # fp32 accumulation of k products: |error| <= ~k * 2^-24 * sum|a_i b_i|
    scale = np.abs(ta.float().cpu().numpy()) @ np.abs(tb.float().cpu().numpy()).T
    assert np.all(np.abs(got - want) <= 1e-6 + (k + 2) * 2.0 ** -23 * (scale + 1e-30))


def test_gemm_rejects_bad_shapes():
    t = torch.zeros((4, 4), dtype=torch.bfloat16, device="cuda")
    o = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(mmas.MMASError, match="n <= 128"):
        mmas.mmas_gemm_bf16(t.data_ptr(), 4, t.data_ptr(), 4, None, o.data_ptr(), 4, 4, 129, 4)


@pytest.mark.parametrize("m,n,k", [
    (64, 64, 2000),     # a weight gradient's shape: 64 x 64, K = n (32 K blocks over 16 CTAs)
    (128, 128, 3000),   # 128 x 128, K = 3000 (ragged last block)
    (200, 64, 130),     # two row tiles, three K blocks
    (8, 64, 18500),     # the input layer's weight gradient at n = 18,500
])
def test_split_k_accumulating_gemm_matches_exact_product(m, n, k):
    # out += A B^T with K split over CTAs (fp32 atomic adds of the partial tiles)
    rng = np.random.default_rng(m + n + k)
    a = rng.standard_normal((m, k)).astype(np.float32)
    b = rng.standard_normal((n, k)).astype(np.float32)
    ta, tb = _bf16(a).cuda(), _bf16(b).cuda()
    out0 = rng.standard_normal((m, n)).astype(np.float32)
    out = torch.from_numpy(out0).cuda()
    mmas.mmas_gemm_bf16_acc(ta.data_ptr(), k, tb.data_ptr(), k, out.data_ptr(), n, m, n, k)
    want = out0.astype(np.float64) + ta.float().cpu().numpy().astype(np.float64) @ \
        tb.float().cpu().numpy().astype(np.float64).T
    got = out.cpu().numpy()
    scale = np.abs(ta.float().cpu().numpy()) @ np.abs(tb.float().cpu().numpy()).T + np.abs(out0)
    # fp32 accumulation inside each split and the atomic adds of the splits
    assert np.all(np.abs(got - want) <= 1e-6 + (k + 64) * 2.0 ** -23 * (scale + 1e-30))
