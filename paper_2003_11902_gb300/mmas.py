"""Python binding of libmmas.so (declared in include/mmas.h).

Argument marshalling only: every step of the MMAS hot path runs in the CUDA
library.  The functions keep the C ABI's names (``mmas_create``,
``mmas_iterate``, ...); ``Colony`` wraps a handle for convenience.  PyTorch, when
importable, supplies the CUDA stream (its current stream) and nothing else.

If the library has not been built, every call raises ``RuntimeError``; there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmmas.so")

MMAS_OK, MMAS_EINVAL, MMAS_ENOMEM, MMAS_ECUDA, MMAS_EOVERFLOW, MMAS_ETIMEOUT, MMAS_ESTATE = range(7)
STATUS_NAMES = {0: "MMAS_OK", 1: "MMAS_EINVAL", 2: "MMAS_ENOMEM", 3: "MMAS_ECUDA",
                4: "MMAS_EOVERFLOW", 5: "MMAS_ETIMEOUT", 6: "MMAS_ESTATE"}

# Every symbol include/mmas.h declares.
EXPORTS = ["mmas_default_params", "mmas_create", "mmas_iterate", "mmas_best_tour",
           "mmas_destroy", "mmas_last_error", "mmas_construct", "mmas_update",
           "mmas_get_tours", "mmas_get_pheromone", "mmas_set_pheromone", "mmas_get_setup",
           "mmas_set_iteration", "mmas_stats", "mmas_synchronize", "mmas_enable_phase_timing",
           "mmas_debug_fail_allocation", "mmas_debug_expire_stage_waits", "mmas_debug_two_opt_move_cap",
           "mmas_shard_best_key", "mmas_shard_tour", "mmas_update_device", "mmas_two_opt_tour",
           "mmas_phase_times", "mmas_score_tours_noalloc", "mmas_probe_draw_rate", "mmas_gemm_bf16",
           "mmas_probe_l2_bandwidth", "mmas_gemm_bf16_acc", "mmas_debug_draw_log2_error",
           "mmas_prior_create", "mmas_prior_set_params", "mmas_prior_get_params",
           "mmas_prior_scores", "mmas_prior_train", "mmas_prior_grad", "mmas_prior_apply",
           "mmas_prior_destroy", "mmas_prior_last_error", "mmas_prior_apply_weighted",
           "mmas_prior_get_state", "mmas_prior_set_state",
           "mmas_batch_create", "mmas_batch_iterate", "mmas_batch_best_tour",
           "mmas_batch_best_lengths", "mmas_batch_get_tours", "mmas_batch_set_config",
           "mmas_batch_get_config", "mmas_batch_autotune", "mmas_batch_synchronize",
           "mmas_batch_enable_phase_timing", "mmas_batch_phase_times", "mmas_batch_fallback_steps",
           "mmas_batch_destroy", "mmas_batch_last_error", "mmas_batch_colony"]
MMAS_NOALLOC_MAX_ANTS = 1048576


class mmas_instance(C.Structure):
    _fields_ = [("n", C.c_int32), ("xy", C.POINTER(C.c_int32)), ("dist", C.POINTER(C.c_int32))]


class mmas_params(C.Structure):
    _fields_ = [("m", C.c_int32), ("alpha", C.c_float), ("beta", C.c_float), ("rho", C.c_float),
                ("p_best", C.c_float), ("cl", C.c_int32), ("seed", C.c_uint64),
                ("deposit", C.c_int32), ("fallback", C.c_int32), ("device", C.c_int32),
                ("ant_offset", C.c_int32), ("ls", C.c_int32), ("selection", C.c_int32),
                ("tabu", C.c_int32), ("stream", C.c_void_p)]


class mmas_batch_config(C.Structure):
    _fields_ = [("warps_per_cta", C.c_int32), ("ctas_per_sm", C.c_int32)]


class mmas_stats_t(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("fallback_steps", C.c_int64), ("nn_len", C.c_int64),
                ("best_len", C.c_int32), ("iter_best_len", C.c_int32), ("tau_min", C.c_float),
                ("tau_max", C.c_float), ("construct_grid", C.c_int32),
                ("construct_block", C.c_int32), ("construct_staged", C.c_int32),
                ("construct_smem", C.c_int32), ("row_pitch", C.c_int32),
                ("fallback_scans", C.c_int64)]


class MMASError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libmmas.so (once) and declare its signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built; run __graft_entry__.build() first")
        L = C.CDLL(path)
        H = C.c_void_p
        P = C.POINTER
        i32, i64, f32 = C.c_int32, C.c_int64, C.c_float
        sigs = {
            "mmas_default_params": (None, [P(mmas_params)]),
            "mmas_create": (C.c_int, [P(mmas_instance), P(mmas_params), P(H)]),
            "mmas_iterate": (C.c_int, [H, i32]),
            "mmas_best_tour": (C.c_int, [H, P(i32), P(i32)]),
            "mmas_destroy": (None, [H]),
            "mmas_last_error": (C.c_char_p, [H]),
            "mmas_construct": (C.c_int, [H]),
            "mmas_update": (C.c_int, [H, P(i32), i32]),
            "mmas_get_tours": (C.c_int, [H, P(i32), P(i32)]),
            "mmas_get_pheromone": (C.c_int, [H, P(f32), P(f32), P(f32)]),
            "mmas_set_pheromone": (C.c_int, [H, P(f32), f32, f32]),
            "mmas_get_setup": (C.c_int, [H, P(i32), P(f32), P(i32), P(i64)]),
            "mmas_set_iteration": (C.c_int, [H, i32]),
            "mmas_stats": (C.c_int, [H, P(mmas_stats_t)]),
            "mmas_debug_fail_allocation": (None, [i32]),
            "mmas_shard_best_key": (C.c_int, [H, C.c_void_p]),
            "mmas_shard_tour": (C.c_int, [H, C.c_void_p, C.c_void_p]),
            "mmas_update_device": (C.c_int, [H, C.c_void_p, C.c_void_p]),
            "mmas_two_opt_tour": (C.c_int, [H, P(i32), P(i32)]),
            "mmas_debug_expire_stage_waits": (C.c_int, [i32, i32]),
            "mmas_debug_two_opt_move_cap": (C.c_int, [i32, i64]),
            "mmas_synchronize": (C.c_int, [H]),
            "mmas_enable_phase_timing": (C.c_int, [H, i32]),
            "mmas_phase_times": (C.c_int, [H, P(f32), P(f32), P(f32)]),
            "mmas_score_tours_noalloc": (C.c_int, [C.c_void_p, i32, i32, i32, C.c_void_p,
                                                  C.c_void_p, C.c_void_p, C.c_void_p]),
            "mmas_probe_draw_rate": (C.c_int, [i32, f32, P(C.c_double)]),
            "mmas_debug_draw_log2_error": (C.c_int, [i32, P(C.c_double), P(C.c_double)]),
            "mmas_probe_l2_bandwidth": (C.c_int, [i32, i64, P(C.c_double)]),
            "mmas_gemm_bf16_acc": (C.c_int, [C.c_void_p, i32, C.c_void_p, i32, C.c_void_p, i32, i32, i32, i32,
                                            C.c_void_p]),
            "mmas_gemm_bf16": (C.c_int, [C.c_void_p, i32, C.c_void_p, i32, C.c_void_p, C.c_void_p,
                                        i32, i32, i32, i32, i32, C.c_void_p]),
            "mmas_prior_create": (C.c_int, [P(f32), i32, P(H)]),
            "mmas_prior_set_params": (C.c_int, [H, P(f32)]),
            "mmas_prior_get_params": (C.c_int, [H, P(f32)]),
            "mmas_prior_get_state": (C.c_int, [H, P(f32), P(f32), P(f32), P(i32)]),
            "mmas_prior_set_state": (C.c_int, [H, P(f32), P(f32), i32]),
            "mmas_prior_scores": (C.c_int, [H, H, P(f32)]),
            "mmas_prior_train": (C.c_int, [H, H, P(i32), i32, f32, P(f32)]),
            "mmas_prior_grad": (C.c_int, [H, H, P(i32), P(f32), P(f32)]),
            "mmas_prior_apply": (C.c_int, [H, H]),
            "mmas_prior_apply_weighted": (C.c_int, [H, H, f32]),
            "mmas_prior_destroy": (None, [H]),
            "mmas_prior_last_error": (C.c_char_p, [H]),
            "mmas_batch_create": (C.c_int, [P(mmas_instance), i32, P(mmas_params), P(H)]),
            "mmas_batch_iterate": (C.c_int, [H, i32]),
            "mmas_batch_best_tour": (C.c_int, [H, i32, P(i32), P(i32)]),
            "mmas_batch_best_lengths": (C.c_int, [H, P(i32)]),
            "mmas_batch_get_tours": (C.c_int, [H, i32, P(i32), P(i32)]),
            "mmas_batch_set_config": (C.c_int, [H, P(mmas_batch_config)]),
            "mmas_batch_get_config": (C.c_int, [H, P(mmas_batch_config)]),
            "mmas_batch_autotune": (C.c_int, [H, i32, P(mmas_batch_config)]),
            "mmas_batch_synchronize": (C.c_int, [H]),
            "mmas_batch_enable_phase_timing": (C.c_int, [H, i32]),
            "mmas_batch_phase_times": (C.c_int, [H, P(f32), P(f32), P(f32)]),
            "mmas_batch_fallback_steps": (C.c_int, [H, P(i64)]),
            "mmas_batch_destroy": (None, [H]),
            "mmas_batch_last_error": (C.c_char_p, [H]),
            "mmas_batch_colony": (C.c_int, [H, i32, P(H)]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _i32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _check(h, status):
    if status != MMAS_OK:
        msg = load().mmas_last_error(h)
        raise MMASError(status, msg.decode() if msg else "")


CUDA_STREAM_LEGACY = 1  # the value of cudaStreamLegacy


def _torch_stream():
    """PyTorch's current stream as a cudaStream_t value.  Its default stream has
    handle 0, which the C ABI reads as "make a private stream", so it is passed
    as cudaStreamLegacy to keep the library ordered with PyTorch's work."""
    try:
        import torch
        if torch.cuda.is_available():
            h = torch.cuda.current_stream().cuda_stream
            return h if h else CUDA_STREAM_LEGACY
    except Exception:
        pass
    return None


# ------------------------------------------------------------- C-named wrappers

def mmas_default_params() -> mmas_params:
    p = mmas_params()
    load().mmas_default_params(C.byref(p))
    return p


def mmas_create(xy=None, dist=None, params: mmas_params | None = None):
    """Create a colony; returns (handle, keep-alive tuple).  Raises MMASError."""
    if (xy is None) == (dist is None):
        raise ValueError("give exactly one of xy and dist")
    p = params if params is not None else mmas_default_params()
    inst = mmas_instance()
    keep = []
    if xy is not None:
        a = np.ascontiguousarray(xy, dtype=np.int32)
        inst.n, inst.xy = a.shape[0], _i32p(a)
        keep.append(a)
    else:
        a = np.ascontiguousarray(dist, dtype=np.int32)
        inst.n, inst.dist = a.shape[0], _i32p(a)
        keep.append(a)
    h = C.c_void_p()
    st = load().mmas_create(C.byref(inst), C.byref(p), C.byref(h))
    _check(None, st)
    return h


def mmas_iterate(h, k: int = 1):
    _check(h, load().mmas_iterate(h, k))


def mmas_best_tour(h, n: int):
    tour = np.zeros(n, np.int32)
    length = C.c_int32()
    _check(h, load().mmas_best_tour(h, _i32p(tour), C.byref(length)))
    return length.value, tour


def mmas_destroy(h):
    load().mmas_destroy(h)


def mmas_last_error(h=None) -> str:
    msg = load().mmas_last_error(h)
    return msg.decode() if msg else ""


def mmas_construct(h):
    _check(h, load().mmas_construct(h))


def mmas_update(h, tour, length: int):
    t = np.ascontiguousarray(tour, dtype=np.int32)
    _check(h, load().mmas_update(h, _i32p(t), int(length)))


def mmas_get_tours(h, m: int, n: int):
    tours = np.zeros((m, n), np.int32)
    lens = np.zeros(m, np.int32)
    _check(h, load().mmas_get_tours(h, _i32p(tours), _i32p(lens)))
    return tours, lens


def mmas_get_pheromone(h, n: int):
    tau = np.zeros((n, n), np.float32)
    tmin, tmax = C.c_float(), C.c_float()
    _check(h, load().mmas_get_pheromone(h, _f32p(tau), C.byref(tmin), C.byref(tmax)))
    return tau, np.float32(tmin.value), np.float32(tmax.value)


def mmas_set_pheromone(h, tau, tmin, tmax):
    t = np.ascontiguousarray(tau, dtype=np.float32)
    _check(h, load().mmas_set_pheromone(h, _f32p(t), float(tmin), float(tmax)))


def mmas_get_setup(h, n: int, cl: int):
    dist = np.zeros((n, n), np.int32)
    eb = np.zeros((n, n), np.float32)
    cand = np.zeros((n, max(cl, 1)), np.int32)
    nn_len = C.c_int64()
    _check(h, load().mmas_get_setup(h, _i32p(dist), _f32p(eb), _i32p(cand), C.byref(nn_len)))
    return dist, eb, cand[:, :cl], nn_len.value


def mmas_set_iteration(h, it: int):
    _check(h, load().mmas_set_iteration(h, int(it)))


def mmas_stats(h) -> dict:
    s = mmas_stats_t()
    _check(h, load().mmas_stats(h, C.byref(s)))
    return {f: getattr(s, f) for f, _ in mmas_stats_t._fields_}


def mmas_debug_fail_allocation(after: int):
    """Arm a simulated device out-of-memory `after` allocations from now
    (-1 disarms); see include/mmas.h."""
    load().mmas_debug_fail_allocation(int(after))


def mmas_debug_expire_stage_waits(device: int, on: bool):
    """Make the construction's staging waits on `device` run out (testing aid;
    see include/mmas.h)."""
    _check(None, load().mmas_debug_expire_stage_waits(int(device), int(bool(on))))


def mmas_debug_two_opt_move_cap(device: int, cap: int):
    """Replace the 2-opt search's move cap on `device` (cap <= 0: the default);
    a testing aid, see include/mmas.h."""
    _check(None, load().mmas_debug_two_opt_move_cap(int(device), int(cap)))


def mmas_synchronize(h):
    _check(h, load().mmas_synchronize(h))


def mmas_enable_phase_timing(h, enable: bool = True):
    _check(h, load().mmas_enable_phase_timing(h, 1 if enable else 0))


def mmas_phase_times(h):
    """(construct_ms, rest_ms, total_ms) of the last timed iteration."""
    a, b, c = C.c_float(), C.c_float(), C.c_float()
    _check(h, load().mmas_phase_times(h, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def mmas_score_tours_noalloc(d_tours: int, m: int, n: int, pitch: int, d_xy: int, d_lens: int,
                             d_best: int, stream=None):
    """Allocation-free scoring of m device-resident tours (device addresses as
    ints, e.g. from torch's data_ptr()): lengths into d_lens, {shortest length,
    its lowest ant} into d_best.  Asynchronous on ``stream`` (a cudaStream_t
    value; None uses PyTorch's current stream when available)."""
    if stream is None:
        stream = _torch_stream()
    _check(None, load().mmas_score_tours_noalloc(d_tours, m, n, pitch, d_xy, d_lens, d_best,
                                                  stream))


def _dptr(x) -> int:
    """A device address: an int, or a tensor's data_ptr()."""
    return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)


# ------------------------------------------------------------------- Colony

class Colony:
    """One MMAS colony on the GPU (a handle of libmmas.so)."""

    def __init__(self, xy=None, dist=None, m=None, alpha=1.0, beta=2.0, rho=0.02, p_best=0.01,
                 cl=32, seed=1, deposit=0, fallback=0, device=0, ant_offset=0, ls=0,
                 selection=0, tabu=0, stream="torch"):
        p = mmas_default_params()
        n = (np.asarray(xy) if xy is not None else np.asarray(dist)).shape[0]
        p.m = int(m) if m is not None else n
        p.alpha, p.beta, p.rho, p.p_best = alpha, beta, rho, p_best
        p.cl, p.seed, p.deposit, p.fallback, p.device = cl, int(seed), deposit, fallback, device
        p.ant_offset = int(ant_offset)
        p.ls = int(ls)
        p.selection, p.tabu = int(selection), int(tabu)
        if stream == "torch":
            stream = _torch_stream()
        elif stream == 0:
            stream = CUDA_STREAM_LEGACY
        p.stream = stream
        self.n, self.m, self.cl = n, p.m, cl
        self.ant_offset = int(ant_offset)
        self._h = mmas_create(xy=xy, dist=dist, params=p)

    @classmethod
    def _borrowed(cls, h, n, m, cl, owner):
        # a handle owned by `owner` (a Batch): close() only drops the reference
        self = cls.__new__(cls)
        self.n, self.m, self.cl, self.ant_offset = n, m, cl, 0
        self._h = h
        self._owner = owner
        return self

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owner", None) is None:
                mmas_destroy(self._h)
            self._h = None
            self._owner = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def iterate(self, k: int = 1):
        mmas_iterate(self._h, k)

    def construct(self):
        mmas_construct(self._h)

    def update(self, tour, length):
        mmas_update(self._h, tour, length)

    def best_tour(self):
        return mmas_best_tour(self._h, self.n)

    def tours(self):
        return mmas_get_tours(self._h, self.m, self.n)

    def pheromone(self):
        return mmas_get_pheromone(self._h, self.n)

    def set_pheromone(self, tau, tmin, tmax):
        mmas_set_pheromone(self._h, tau, tmin, tmax)

    def setup(self):
        d, eb, cand, nn_len = mmas_get_setup(self._h, self.n, self.cl)
        return {"d": d, "eta_beta": eb, "cand": cand, "nn_len": nn_len}

    def set_iteration(self, it: int):
        mmas_set_iteration(self._h, it)

    def stats(self) -> dict:
        return mmas_stats(self._h)

    def two_opt(self, tour):
        """The colony's 2-opt applied to a copy of `tour`: (improved tour, length)."""
        t = np.array(tour, dtype=np.int32, copy=True, order="C")
        n = C.c_int32()
        _check(self._h, load().mmas_two_opt_tour(self._h, _i32p(t), C.byref(n)))
        return t, n.value

    def shard_best_key(self, key):
        """Enqueue: the device int64 `key` (a tensor or an address) = (length
        << 32 | global ant) of the shortest tour of the last construction."""
        _check(self._h, load().mmas_shard_best_key(self._h, _dptr(key)))

    def shard_tour(self, key, tour):
        """Enqueue: device int32[n] `tour` = the key's tour if this shard built
        it, else zeros."""
        _check(self._h, load().mmas_shard_tour(self._h, _dptr(key), _dptr(tour)))

    def update_device(self, tour, key):
        """Enqueue the update with a device-side tour and the key's length,
        then advance the iteration index."""
        _check(self._h, load().mmas_update_device(self._h, _dptr(tour), _dptr(key)))

    def synchronize(self):
        mmas_synchronize(self._h)

    def enable_phase_timing(self, enable: bool = True):
        mmas_enable_phase_timing(self._h, enable)

    def phase_times(self):
        return mmas_phase_times(self._h)


def mmas_probe_draw_rate(device: int = 0, ms: float = 50.0) -> float:
    """Draws per second of the selection's per-candidate arithmetic at full
    occupancy (a measurement aid; see include/mmas.h)."""
    v = C.c_double()
    _check(None, load().mmas_probe_draw_rate(device, ms, C.byref(v)))
    return v.value


def mmas_debug_draw_log2_error(device: int = 0):
    """(largest relative error of the draws' log2, that of the library's log2f)
    over every draw value (a test hook; see include/mmas.h)."""
    a, b = C.c_double(), C.c_double()
    _check(None, load().mmas_debug_draw_log2_error(device, C.byref(a), C.byref(b)))
    return a.value, b.value


def mmas_probe_l2_bandwidth(device: int = 0, nbytes: int = 32 << 20) -> float:
    """L2 read bandwidth in GB/s over an L2-resident buffer (a measurement aid;
    see include/mmas.h)."""
    v = C.c_double()
    _check(None, load().mmas_probe_l2_bandwidth(device, int(nbytes), C.byref(v)))
    return v.value


def mmas_gemm_bf16(d_a: int, lda: int, d_b: int, ldb: int, d_bias, d_out: int, ldd: int,
                   m: int, n: int, k: int, relu: bool = False, stream=None):
    """out = act(A B^T + bias) on the tensor cores; every pointer is a device
    address (e.g. a torch tensor's data_ptr()); see include/mmas.h."""
    if stream is None:
        stream = _torch_stream()
    _check(None, load().mmas_gemm_bf16(d_a, lda, d_b, ldb, d_bias, d_out, ldd, m, n, k,
                                       int(relu), stream))


def mmas_gemm_bf16_acc(d_a: int, lda: int, d_b: int, ldb: int, d_out: int, ldd: int, m: int, n: int, k: int,
                       stream=None):
    """out += A B^T on the tensor cores with K split over CTAs (device
    addresses); see include/mmas.h."""
    if stream is None:
        stream = _torch_stream()
    _check(None, load().mmas_gemm_bf16_acc(d_a, lda, d_b, ldb, d_out, ldd, m, n, k, stream))


# ------------------------------------------------------------------- learned prior

MMAS_PRIOR_PARAMS = 29442


def _pcheck(p, status):
    if status != MMAS_OK:
        msg = load().mmas_prior_last_error(p)
        raise MMASError(status, msg.decode() if msg else "")


class Prior:
    """The learned edge prior (see include/mmas.h): a message-passing network
    whose edge probabilities can replace a colony's eta^beta."""

    def __init__(self, params=None, device=0):
        h = C.c_void_p()
        if params is not None:
            params = np.ascontiguousarray(params, dtype=np.float32)
            assert params.size == MMAS_PRIOR_PARAMS
        _pcheck(None, load().mmas_prior_create(_f32p(params) if params is not None else None, device,
                                               C.byref(h)))
        self._p = h

    def close(self):
        if getattr(self, "_p", None):
            load().mmas_prior_destroy(self._p)
            self._p = None

    __del__ = close

    def set_params(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32)
        _pcheck(self._p, load().mmas_prior_set_params(self._p, _f32p(params)))

    def params(self):
        out = np.zeros(MMAS_PRIOR_PARAMS, np.float32)
        _pcheck(self._p, load().mmas_prior_get_params(self._p, _f32p(out)))
        return out

    def state(self):
        """(m, v, grad, step): Adam's moments, the last gradient and the step count."""
        m = np.zeros(MMAS_PRIOR_PARAMS, np.float32)
        v = np.zeros(MMAS_PRIOR_PARAMS, np.float32)
        g = np.zeros(MMAS_PRIOR_PARAMS, np.float32)
        t = C.c_int32()
        _pcheck(self._p, load().mmas_prior_get_state(self._p, _f32p(m), _f32p(v), _f32p(g), C.byref(t)))
        return m, v, g, t.value

    def set_state(self, m, v, step: int):
        m = np.ascontiguousarray(m, dtype=np.float32)
        v = np.ascontiguousarray(v, dtype=np.float32)
        _pcheck(self._p, load().mmas_prior_set_state(self._p, _f32p(m), _f32p(v), int(step)))

    def scores(self, colony: "Colony"):
        out = np.zeros((colony.n, 16), np.float32)
        _pcheck(self._p, load().mmas_prior_scores(self._p, colony._h, _f32p(out)))
        return out

    def train(self, colony: "Colony", tour, steps: int = 1, lr: float = 1e-3) -> float:
        t = np.ascontiguousarray(tour, dtype=np.int32)
        loss = C.c_float()
        _pcheck(self._p, load().mmas_prior_train(self._p, colony._h, _i32p(t), steps, lr, C.byref(loss)))
        return loss.value

    def grad(self, colony: "Colony", tour):
        t = np.ascontiguousarray(tour, dtype=np.int32)
        g = np.zeros(MMAS_PRIOR_PARAMS, np.float32)
        loss = C.c_float()
        _pcheck(self._p, load().mmas_prior_grad(self._p, colony._h, _i32p(t), _f32p(g), C.byref(loss)))
        return g, loss.value

    def apply(self, colony: "Colony"):
        _pcheck(self._p, load().mmas_prior_apply(self._p, colony._h))

    def apply_weighted(self, colony: "Colony", gamma: float = 1.0):
        _pcheck(self._p, load().mmas_prior_apply_weighted(self._p, colony._h, float(gamma)))


# ------------------------------------------------------------------- batches

def _bcheck(b, status):
    if status != MMAS_OK:
        msg = load().mmas_batch_last_error(b)
        raise MMASError(status, msg.decode() if msg else "")


def mmas_batch_create(instances, params: mmas_params):
    """instances: list of (xy or None, dist or None) int32 arrays; returns the handle."""
    arr = (mmas_instance * len(instances))()
    keep = []
    for i, (xy, dist) in enumerate(instances):
        if (xy is None) == (dist is None):
            raise ValueError("give exactly one of xy and dist per instance")
        a = np.ascontiguousarray(xy if xy is not None else dist, dtype=np.int32)
        keep.append(a)
        arr[i].n = a.shape[0]
        if xy is not None:
            arr[i].xy = _i32p(a)
        else:
            arr[i].dist = _i32p(a)
    b = C.c_void_p()
    _bcheck(None, load().mmas_batch_create(arr, len(instances), C.byref(params), C.byref(b)))
    return b


class Batch:
    """Many colonies advanced together (batched launches; see include/mmas.h).
    Colony c uses seed + c and m = m or n_c."""

    def __init__(self, xys=None, dists=None, m=0, alpha=1.0, beta=2.0, rho=0.02, p_best=0.01,
                 cl=32, seed=1, deposit=0, fallback=0, device=0, stream="torch"):
        if (xys is None) == (dists is None):
            raise ValueError("give exactly one of xys and dists")
        insts = [(x, None) for x in xys] if xys is not None else [(None, d) for d in dists]
        p = mmas_default_params()
        p.m = int(m)
        p.alpha, p.beta, p.rho, p.p_best = alpha, beta, rho, p_best
        p.cl, p.seed, p.deposit, p.fallback, p.device = cl, int(seed), deposit, fallback, device
        if stream == "torch":
            stream = _torch_stream()
        elif stream == 0:
            stream = CUDA_STREAM_LEGACY
        p.stream = stream
        self.ns = [np.asarray(x if x is not None else d).shape[0] for x, d in insts]
        self.ms = [int(m) if m else n for n in self.ns]
        self.cl = cl
        self._b = mmas_batch_create(insts, p)

    def close(self):
        if getattr(self, "_b", None):
            load().mmas_batch_destroy(self._b)
            self._b = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __len__(self):
        return len(self.ns)

    def iterate(self, k: int = 1):
        _bcheck(self._b, load().mmas_batch_iterate(self._b, k))

    def best_tour(self, c: int):
        tour = np.zeros(self.ns[c], np.int32)
        length = C.c_int32()
        _bcheck(self._b, load().mmas_batch_best_tour(self._b, c, _i32p(tour), C.byref(length)))
        return length.value, tour

    def colony(self, c: int) -> "Colony":
        """Colony c as a Colony object sharing the batch's state (owned by the batch)."""
        h = C.c_void_p()
        _bcheck(self._b, load().mmas_batch_colony(self._b, int(c), C.byref(h)))
        return Colony._borrowed(h, self.ns[c], self.ms[c], self.cl, self)

    def best_lengths(self):
        out = np.zeros(len(self.ns), np.int32)
        _bcheck(self._b, load().mmas_batch_best_lengths(self._b, _i32p(out)))
        return out

    def tours(self, c: int):
        t = np.zeros((self.ms[c], self.ns[c]), np.int32)
        lens = np.zeros(self.ms[c], np.int32)
        _bcheck(self._b, load().mmas_batch_get_tours(self._b, c, _i32p(t), _i32p(lens)))
        return t, lens

    def set_config(self, warps_per_cta: int, ctas_per_sm: int):
        cfg = mmas_batch_config(warps_per_cta, ctas_per_sm)
        _bcheck(self._b, load().mmas_batch_set_config(self._b, C.byref(cfg)))

    def config(self):
        cfg = mmas_batch_config()
        _bcheck(self._b, load().mmas_batch_get_config(self._b, C.byref(cfg)))
        return cfg.warps_per_cta, cfg.ctas_per_sm

    def autotune(self, reps: int = 3):
        cfg = mmas_batch_config()
        _bcheck(self._b, load().mmas_batch_autotune(self._b, reps, C.byref(cfg)))
        return cfg.warps_per_cta, cfg.ctas_per_sm

    def synchronize(self):
        _bcheck(self._b, load().mmas_batch_synchronize(self._b))

    def enable_phase_timing(self, enable: bool = True):
        _bcheck(self._b, load().mmas_batch_enable_phase_timing(self._b, int(enable)))

    def phase_times(self):
        a, b, t = C.c_float(), C.c_float(), C.c_float()
        _bcheck(self._b, load().mmas_batch_phase_times(self._b, C.byref(a), C.byref(b), C.byref(t)))
        return a.value, b.value, t.value

    def fallback_steps(self) -> int:
        v = C.c_int64()
        _bcheck(self._b, load().mmas_batch_fallback_steps(self._b, C.byref(v)))
        return v.value
