"""Failure paths of the library, made on the host or by a bounded device wait
that is made to run out -- never by faulting the GPU:
  - a tour-length overflow (n * max distance >= 2^31) refused with EOVERFLOW;
  - a simulated device out-of-memory at every allocation of mmas_create,
    mmas_batch_create and the learned prior: ENOMEM, nothing left allocated;
  - the construction's staging wait made to run out: ETIMEOUT at the next
    synchronising call, and the device stays usable;
  - the 2-opt search's move cap made small enough to be hit: ESTATE, the
    tours still permutations."""
import numpy as np
import pytest

import oracle as O
from paper_2003_11902_gb300 import Batch, Colony, MMASError, Prior, instances as I
from paper_2003_11902_gb300 import mmas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    yield
    mmas.mmas_debug_fail_allocation(-1)
    mmas.mmas_debug_expire_stage_waits(0, False)
    mmas.mmas_debug_two_opt_move_cap(0, 0)


def test_tour_length_overflow_is_refused():
    # three coordinates whose longest distance is about 1.5e9: 3 x 1.5e9 >= 2^31
    big = (1 << 30) - 1
    xy = np.array([[0, 0], [big, 0], [0, big]], np.int32)
    with pytest.raises(MMASError) as e:
        Colony(xy=xy, m=2, cl=0)
    assert e.value.status == mmas.MMAS_EOVERFLOW
    # the same through an explicit matrix, and one just below the limit passes
    d = np.full((3, 3), 1 << 30, np.int32)
    np.fill_diagonal(d, 0)
    with pytest.raises(MMASError) as e:
        Colony(dist=d, m=2, cl=0)
    assert e.value.status == mmas.MMAS_EOVERFLOW
    d = np.full((3, 3), (1 << 31) // 3 - 1, np.int32)
    np.fill_diagonal(d, 0)
    with Colony(dist=d, m=2, cl=0) as g:
        g.iterate(1)
        assert g.best_tour()[0] == 3 * ((1 << 31) // 3 - 1)


def _free():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _fail_each_allocation(make, limit=400):
    """Arm a failure at allocation 0, 1, 2, ... of make() until one succeeds;
    every failed call raises ENOMEM.  Returns how many allocations were hit."""
    for k in range(limit):
        mmas.mmas_debug_fail_allocation(k)
        try:
            obj = make()
        except MMASError as e:
            assert e.status == mmas.MMAS_ENOMEM, e
            continue
        finally:
            mmas.mmas_debug_fail_allocation(-1)
        obj.close()
        return k
    raise AssertionError("the call never got past its allocations")


def test_out_of_memory_in_create_leaves_nothing_behind():
    xy = I.uniform(300, 3)
    Colony(xy=xy, m=64, cl=16).close()  # warm the allocator and the module
    before = _free()
    hit = _fail_each_allocation(lambda: Colony(xy=xy, m=64, cl=16, ls=1))
    assert hit >= 10  # every buffer of the colony was a failure point
    assert abs(_free() - before) <= (8 << 20)
    with Colony(xy=xy, m=64, cl=16, ls=1) as g:  # a normal create still works
        g.iterate(2)
        assert g.best_tour()[0] > 0


def test_out_of_memory_in_batch_create_and_prior():
    xys = [I.uniform(n, 10 + n) for n in (60, 130, 90)]
    Batch(xys=xys, cl=16).close()
    before = _free()
    hit = _fail_each_allocation(lambda: Batch(xys=xys, cl=16))
    assert hit >= 3 * 10
    assert abs(_free() - before) <= (8 << 20)
    with Colony(xy=I.uniform(200, 4), m=8, cl=16) as col:
        class Scored:  # the prior allocates its workspace at its first use on a colony
            def __init__(self):
                self.p = Prior(I.prior_params(1))
                try:
                    self.s = self.p.scores(col)
                except Exception:
                    self.p.close()
                    raise

            def close(self):
                self.p.close()
        hit = _fail_each_allocation(Scored)
        assert hit >= 10
    assert abs(_free() - before) <= (8 << 20)


def test_staging_wait_that_runs_out_reports_a_timeout():
    xy = I.uniform(1000, 1001)
    g = Colony(xy=xy, m=200, cl=32, seed=1)
    assert g.stats()["construct_staged"] == 1
    mmas.mmas_debug_expire_stage_waits(0, True)
    try:
        g.iterate(1)
        with pytest.raises(MMASError) as e:
            g.synchronize()
        assert e.value.status == mmas.MMAS_ETIMEOUT
    finally:
        mmas.mmas_debug_expire_stage_waits(0, False)
    g.close()
    # the device is still usable: a fresh colony matches the oracle
    g = Colony(xy=I.uniform(64, 7), m=64, cl=16, rho=0.1, seed=3)
    o = O.Colony(xy=I.uniform(64, 7), m=64, cl=16, rho=0.1, seed=3, p_best=float(np.float32(0.01)))
    g.iterate(1)
    o.iterate(1)
    assert np.array_equal(g.tours()[0], o.tours()[0])
    g.close()


def test_two_opt_move_cap_reports_a_state_error():
    xy = I.uniform(400, 21)
    g = Colony(xy=xy, m=32, cl=16, seed=4, ls=2)
    mmas.mmas_debug_two_opt_move_cap(0, 3)
    try:
        g.iterate(1)
        with pytest.raises(MMASError, match="move cap") as e:
            g.synchronize()
        assert e.value.status == mmas.MMAS_ESTATE
    finally:
        mmas.mmas_debug_two_opt_move_cap(0, 0)
    tours, _ = g.tours()
    assert all(sorted(t) == list(range(400)) for t in tours)  # stopped searches keep whole tours
    g.iterate(1)
    g.synchronize()  # the default cap: no error
    g.close()
