"""The C ABI library builds, loads and exports every symbol include/mmas.h
declares; parameter validation happens on the host before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2003_11902_gb300 import _build, instances, mmas

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return mmas.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "mmas.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mmas_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) == 57
    assert sorted(mmas.EXPORTS) == declared
    for name in declared:
        assert hasattr(lib, name), name


def test_struct_layout_matches_header():
    assert C.sizeof(mmas.mmas_params) == 72
    assert mmas.mmas_params.seed.offset == 24
    assert mmas.mmas_params.selection.offset == 52
    assert mmas.mmas_params.stream.offset == 64
    assert C.sizeof(mmas.mmas_instance) == 24
    assert C.sizeof(mmas.mmas_batch_config) == 8


def test_default_params(lib):
    p = mmas.mmas_default_params()
    assert (p.m, p.alpha, p.beta, p.cl, p.seed) == (0, 1.0, 2.0, 32, 1)
    assert abs(p.rho - 0.02) < 1e-7 and abs(p.p_best - 0.01) < 1e-7


@pytest.mark.parametrize("field,value,needle", [
    ("rho", 0.0, "rho"), ("rho", 1.0, "rho"), ("p_best", 1.0, "p_best"), ("alpha", -1.0, "alpha"),
    ("beta", float("nan"), "beta"), ("cl", 65, "cl"), ("cl", -1, "cl"), ("m", -5, "m must"),
    ("deposit", 2, "deposit"), ("fallback", 3, "fallback"), ("ls", 3, "ls"),
    ("selection", 2, "selection"), ("tabu", -1, "tabu"),
])
def test_bad_parameters_are_rejected_before_device_work(lib, field, value, needle):
    p = mmas.mmas_default_params()
    setattr(p, field, value)
    with pytest.raises(mmas.MMASError) as e:
        mmas.mmas_create(xy=instances.uniform(50, 1), params=p)
    assert e.value.status == mmas.MMAS_EINVAL
    assert needle in str(e.value)
    assert needle in mmas.mmas_last_error(None)


def test_local_search_needs_short_candidate_lists(lib):
    p = mmas.mmas_default_params()
    p.cl, p.ls = 40, 1
    with pytest.raises(mmas.MMASError, match="cl <= 32"):
        mmas.mmas_create(xy=instances.uniform(50, 1), params=p)


def test_bad_instances_are_rejected(lib):
    p = mmas.mmas_default_params()
    p.cl = 2
    with pytest.raises(mmas.MMASError, match="n must be"):
        mmas.mmas_create(xy=instances.uniform(2, 1), params=p)
    d = np.array([[0, 1, 2], [1, 0, 3], [2, 4, 0]], np.int32)
    with pytest.raises(mmas.MMASError, match="symmetric"):
        mmas.mmas_create(dist=d, params=p)
    d = np.array([[0, 1, 2], [1, 1, 3], [2, 3, 0]], np.int32)
    with pytest.raises(mmas.MMASError, match="diagonal"):
        mmas.mmas_create(dist=d, params=p)
    xy = np.array([[0, 0], [1 << 30, 0], [5, 5]], np.int32)
    with pytest.raises(mmas.MMASError, match="2\\^30"):
        mmas.mmas_create(xy=xy, params=p)
    p.cl = 3
    with pytest.raises(mmas.MMASError, match="cl must"):
        mmas.mmas_create(xy=instances.uniform(3, 1), params=p)


def test_missing_library_fails_loudly(tmp_path):
    saved = mmas._lib
    mmas._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            mmas.load(str(tmp_path / "libmmas.so"))
    finally:
        mmas._lib = saved


def test_no_device_is_an_error_not_a_fallback(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(mmas.MMASError) as e:
        mmas.Colony(xy=instances.uniform(20, 1), cl=4, stream=None)
    assert e.value.status == mmas.MMAS_ECUDA


@pytest.mark.parametrize("field,value,needle", [
    ("cl", 0, "1 <= cl <= 32"), ("ls", 1, "local search"), ("ant_offset", 5, "ant_offset"),
])
def test_batch_restrictions_are_checked_first(lib, field, value, needle):
    p = mmas.mmas_default_params()
    setattr(p, field, value)
    with pytest.raises(mmas.MMASError) as e:
        mmas.mmas_batch_create([(instances.uniform(30, 1), None)], p)
    assert e.value.status == mmas.MMAS_EINVAL and needle in str(e.value)
    assert needle in load_batch_error(lib)


def load_batch_error(lib):
    return lib.mmas_batch_last_error(None).decode()


def test_batch_instance_checks(lib):
    p = mmas.mmas_default_params()
    p.cl = 4
    with pytest.raises(mmas.MMASError, match="every instance"):
        mmas.mmas_batch_create([(instances.uniform(30, 1), None),
                                (None, np.zeros((3, 3), np.int32))], p)
    with pytest.raises(mmas.MMASError, match="count >= 1"):
        mmas.mmas_batch_create([], p)
    # colony 0 fails its own validation: the message names it
    with pytest.raises(mmas.MMASError, match="colony 0: n must be"):
        mmas.mmas_batch_create([(instances.uniform(2, 1), None), (instances.uniform(30, 2), None)], p)


def test_whole_row_variants_need_whole_rows(lib):
    p = mmas.mmas_default_params()
    p.cl, p.selection = 8, 1
    with pytest.raises(mmas.MMASError, match="whole-row"):
        mmas.mmas_create(xy=instances.uniform(50, 1), params=p)
