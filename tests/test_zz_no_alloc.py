"""The allocation-free scoring entry point, mmas_score_tours_noalloc.

It exists for callers that cannot let a library allocate device memory:
latency-critical serving loops (cudaMalloc/cudaFree synchronise the device)
and frameworks whose caching allocator owns the memory budget.  Here the test
owns every buffer it passes (PyTorch tensors) and checks, through the C ABI,
that the entry point reproduces the colony's own scoring -- the tour lengths
read back by mmas_get_tours and the iteration best reported by mmas_stats --
exactly, on two calls in a row (the second with padded rows), so the shared
scratch is reset between calls.
"""
import numpy as np
import pytest

from paper_2003_11902_gb300 import Colony, MMASError, instances as I, mmas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_noalloc_scoring_matches_the_colony_on_two_calls():
    torch = pytest.importorskip("torch")
    n, m = 1000, 1000
    xy = I.uniform(n, 1001)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        col = Colony(xy=xy, m=m, cl=32, seed=1)
        d_xy = torch.from_numpy(xy).cuda()
        d_lens = torch.empty(m, dtype=torch.int32, device="cuda")
        d_best = torch.empty(2, dtype=torch.int32, device="cuda")
        for call, pitch in enumerate((n, 1024)):
            col.iterate(1)
            tours, lens = col.tours()
            st = col.stats()
            padded = np.zeros((m, pitch), np.int32)
            padded[:, :n] = tours
            d_tours = torch.from_numpy(padded).cuda()
            d_lens.fill_(-1)
            d_best.fill_(-1)
            mmas.mmas_score_tours_noalloc(d_tours.data_ptr(), m, n, pitch, d_xy.data_ptr(),
                                          d_lens.data_ptr(), d_best.data_ptr(), stream.cuda_stream)
            stream.synchronize()
            got_lens = d_lens.cpu().numpy()
            best = d_best.cpu().numpy()
            assert np.array_equal(got_lens, lens), f"call {call}: lengths differ"
            assert best[0] == st["iter_best_len"] == lens.min(), f"call {call}: best length"
            assert best[1] == int(np.argmin(lens)), f"call {call}: best ant"
    col.close()


def test_noalloc_rejects_sizes_beyond_its_limits():
    for m, n, pitch in [(mmas.MMAS_NOALLOC_MAX_ANTS + 1, 100, 100), (0, 100, 100),
                        (10, 2, 2), (10, 100, 99)]:
        with pytest.raises(MMASError) as e:
            mmas.mmas_score_tours_noalloc(16, m, n, pitch, 16, 16, 16, None)
        assert e.value.status == mmas.MMAS_EINVAL
        assert "mmas_score_tours_noalloc" in mmas.mmas_last_error(None)
