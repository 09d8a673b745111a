"""Python access to the CPU oracle (``mmas_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are its only users. The CUDA library never calls it.

``build()`` compiles the C file with gcc (no CUDA, no shared code with the GPU
path); ``lib()`` loads it. The wrappers below only marshal numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mmas_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the source (gcc, -O2, OpenMP, no FP contraction)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _i32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _f64p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i64p(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            vp, i32, i64, u32, u64, f32, f64 = (C.c_void_p, C.c_int32, C.c_int64, C.c_uint32,
                                                C.c_uint64, C.c_float, C.c_double)
            P = C.POINTER
            sig = {
                "orc_philox4x32_10": (None, [P(u32), P(u32), P(u32)]),
                "orc_uniform01": (f64, [u32]),
                "orc_word_start": (u32, [u64, i32, i32]),
                "orc_word_cand": (u32, [u64, i32, i32, i32, i32]),
                "orc_word_row": (u32, [u64, i32, i32, i32, i32]),
                "orc_word_slot": (u32, [u64, i32, i32, i32, i32]),
                "orc_word_rwm": (u32, [u64, i32, i32, i32]),
                "orc_variant_step": (i32, [vp, i32, i32, P(i32), i32, P(i32), P(f64), P(i32),
                                           P(f64)]),
                "orc_colony_set_variant": (None, [vp, i32, i32]),
                "orc_start_node": (i32, [u64, i32, i32, i32]),
                "orc_isqrt64": (u64, [u64]),
                "orc_euc2d": (i64, [i32, i32, i32, i32]),
                "orc_distances": (None, [i32, P(i32), P(i32)]),
                "orc_eta_beta": (None, [i32, P(i32), f64, P(f32)]),
                "orc_candidates": (None, [i32, P(i32), i32, P(i32)]),
                "orc_tour_length": (i64, [i32, P(i32), P(i32)]),
                "orc_nn_tour": (i64, [i32, P(i32), P(i32)]),
                "orc_limits": (None, [i32, f64, f64, i64, P(f32), P(f32)]),
                "orc_choice": (None, [i32, P(f32), P(f32), f64, P(f32)]),
                "orc_evaporate": (None, [i32, P(f32), f32, f32, f32]),
                "orc_deposit": (None, [i32, P(f32), P(i32), f32, f32]),
                "orc_wrs_pick": (i32, [i32, P(i32), P(f64), P(f64)]),
                "orc_rwm_pick": (i32, [i32, P(f64), f64]),
                "orc_colony_new": (vp, [i32, P(i32), P(i32), i32, i32, f64, f64, f32, f64, u64,
                                        i32, i32, i32]),
                "orc_colony_free": (None, [vp]),
                "orc_step_keys": (i32, [vp, i32, i32, i32, i32, P(C.c_uint8), P(f64)]),
                "orc_colony_construct": (i64, [vp, i32, i32, P(i32), P(i64)]),
                "orc_colony_iterate": (None, [vp, i32]),
                "orc_colony_update": (None, [vp, P(i32), i64]),
                "orc_colony_set_pheromone": (None, [vp, P(f32), f32, f32]),
                "orc_colony_iter": (i32, [vp]),
                "orc_colony_nn_len": (i64, [vp]),
                "orc_colony_best": (i64, [vp, P(i32)]),
                "orc_colony_limits": (None, [vp, P(f32), P(f32)]),
                "orc_colony_get": (None, [vp, P(i32), P(f32), P(i32), P(f32), P(f32)]),
                "orc_colony_tours": (None, [vp, P(i32), P(i64), P(i64)]),
                "orc_brute_force": (i64, [i32, P(i32), P(i32)]),
                "orc_two_opt": (i64, [i32, P(i32), P(i32), i32, P(i32)]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


# ---------------------------------------------------------------- primitives

def philox4x32_10(ctr, key):
    ctr = np.asarray(ctr, dtype=np.uint32)
    key = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    P = C.POINTER(C.c_uint32)
    lib().orc_philox4x32_10(ctr.ctypes.data_as(P), key.ctypes.data_as(P), out.ctypes.data_as(P))
    return out


def uniform01(x: int) -> float:
    return lib().orc_uniform01(x)


def word_start(seed, it, ant):
    return lib().orc_word_start(seed, it, ant)


def word_cand(seed, it, ant, t, s):
    return lib().orc_word_cand(seed, it, ant, t, s)


def word_row(seed, it, ant, t, v):
    return lib().orc_word_row(seed, it, ant, t, v)


def start_node(seed, it, ant, n):
    return lib().orc_start_node(seed, it, ant, n)


def isqrt64(s: int) -> int:
    return lib().orc_isqrt64(s)


def euc2d(x1, y1, x2, y2) -> int:
    return lib().orc_euc2d(x1, y1, x2, y2)


def distances(xy):
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    n = xy.shape[0]
    d = np.zeros((n, n), dtype=np.int32)
    lib().orc_distances(n, _i32p(xy), _i32p(d))
    return d


def eta_beta(d, beta):
    d = np.ascontiguousarray(d, dtype=np.int32)
    n = d.shape[0]
    eb = np.zeros((n, n), dtype=np.float32)
    lib().orc_eta_beta(n, _i32p(d), float(beta), _f32p(eb))
    return eb


def candidates(d, cl):
    d = np.ascontiguousarray(d, dtype=np.int32)
    n = d.shape[0]
    cand = np.zeros((n, cl), dtype=np.int32)
    lib().orc_candidates(n, _i32p(d), cl, _i32p(cand))
    return cand


def tour_length(d, tour) -> int:
    d = np.ascontiguousarray(d, dtype=np.int32)
    tour = np.ascontiguousarray(tour, dtype=np.int32)
    return lib().orc_tour_length(d.shape[0], _i32p(d), _i32p(tour))


def nn_tour(d):
    d = np.ascontiguousarray(d, dtype=np.int32)
    n = d.shape[0]
    tour = np.zeros(n, dtype=np.int32)
    length = lib().orc_nn_tour(n, _i32p(d), _i32p(tour))
    return length, tour


def limits(n, rho, p_best, cost):
    tmax = C.c_float()
    tmin = C.c_float()
    lib().orc_limits(n, float(rho), float(p_best), int(cost), C.byref(tmax), C.byref(tmin))
    return np.float32(tmax.value), np.float32(tmin.value)


def choice(tau, eb, alpha):
    tau = np.ascontiguousarray(tau, dtype=np.float32)
    eb = np.ascontiguousarray(eb, dtype=np.float32)
    out = np.zeros_like(tau)
    lib().orc_choice(tau.shape[0], _f32p(tau), _f32p(eb), float(alpha), _f32p(out))
    return out


def evaporate(tau, persist, tmin, tmax):
    tau = np.array(tau, dtype=np.float32, copy=True, order="C")
    lib().orc_evaporate(tau.shape[0], _f32p(tau), np.float32(persist), np.float32(tmin),
                        np.float32(tmax))
    return tau


def deposit(tau, tour, delta, tmax):
    tau = np.array(tau, dtype=np.float32, copy=True, order="C")
    tour = np.ascontiguousarray(tour, dtype=np.int32)
    lib().orc_deposit(tau.shape[0], _f32p(tau), _i32p(tour), np.float32(delta), np.float32(tmax))
    return tau


def persist_factor(rho) -> np.float32:
    """The float 1 - rho by which evaporation multiplies (reading R-rho)."""
    return np.float32(1.0 - float(np.float32(rho)))


def wrs_pick(ids, w, r) -> int:
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    return lib().orc_wrs_pick(len(w), _i32p(ids), _f64p(w), _f64p(r))


def rwm_pick(w, u) -> int:
    """The roulette wheel over weights w with draw u (orc_rwm_pick): the first
    position whose cumulative sum exceeds u * sum(w); -1 if no weight is positive."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    return lib().orc_rwm_pick(len(w), _f64p(w), float(u))


def word_slot(seed, it, ant, t, j):
    return lib().orc_word_slot(seed, it, ant, t, j)


def word_rwm(seed, it, ant, t):
    return lib().orc_word_rwm(seed, it, ant, t)


def two_opt(d, nn, tour):
    """2-opt with neighbour lists nn (n x k) and don't-look bits; returns
    (improved tour, number of moves)."""
    d = np.ascontiguousarray(d, dtype=np.int32)
    nn = np.ascontiguousarray(nn, dtype=np.int32)
    t = np.array(tour, dtype=np.int32, copy=True, order="C")
    moves = lib().orc_two_opt(d.shape[0], _i32p(d), _i32p(nn), nn.shape[1], _i32p(t))
    return t, moves


def brute_force(d):
    d = np.ascontiguousarray(d, dtype=np.int32)
    n = d.shape[0]
    tour = np.zeros(n, dtype=np.int32)
    length = lib().orc_brute_force(n, _i32p(d), _i32p(tour))
    return length, tour


# ---------------------------------------------------------------- the colony

class Colony:
    """The oracle's MMAS (Alg. 1) on one instance; same parameters as the C ABI."""

    def __init__(self, n=None, xy=None, dist=None, m=1, cl=0, alpha=1.0, beta=2.0, rho=0.02,
                 p_best=0.01, seed=1, deposit=0, fallback=0, ls=0, selection=0, tabu=0):
        if (xy is None) == (dist is None):
            raise ValueError("give exactly one of xy and dist")
        if xy is not None:
            self._xy = np.ascontiguousarray(xy, dtype=np.int32)
            n = self._xy.shape[0]
            xyp, dp = _i32p(self._xy), None
        else:
            self._dist = np.ascontiguousarray(dist, dtype=np.int32)
            n = self._dist.shape[0]
            xyp, dp = None, _i32p(self._dist)
        self.n, self.m, self.cl = n, m, cl
        self.seed, self.fallback, self.deposit = seed, fallback, deposit
        if ls and cl < 1:
            raise ValueError("local search uses the candidate lists: cl must be >= 1")
        self.ls = ls
        if (selection or tabu) and cl != 0:
            raise ValueError("the roulette wheel and the compact tabu are whole-row variants (cl = 0)")
        self.selection, self.tabu = selection, tabu
        self._h = lib().orc_colony_new(n, xyp, dp, m, cl, float(alpha), float(beta),
                                       float(np.float32(rho)), float(p_best), int(seed),
                                       deposit, fallback, ls)
        lib().orc_colony_set_variant(self._h, int(selection), int(tabu))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_colony_free(h)
            self._h = None

    @property
    def iteration(self) -> int:
        return lib().orc_colony_iter(self._h)

    @property
    def nn_len(self) -> int:
        return lib().orc_colony_nn_len(self._h)

    def iterate(self, k: int = 1, threads: int = 1):
        for _ in range(k):
            lib().orc_colony_iterate(self._h, threads)

    def update(self, ib_tour, ib_len):
        """Alg. 1 after construction, with a given iteration-best tour."""
        t = np.ascontiguousarray(ib_tour, dtype=np.int32)
        lib().orc_colony_update(self._h, _i32p(t), int(ib_len))

    def set_pheromone(self, tau, tmin, tmax):
        """Start from pheromone `tau` (n x n) and limits; choice_info follows."""
        t = np.ascontiguousarray(tau, dtype=np.float32)
        lib().orc_colony_set_pheromone(self._h, _f32p(t), float(tmin), float(tmax))

    def best(self):
        tour = np.zeros(self.n, dtype=np.int32)
        length = lib().orc_colony_best(self._h, _i32p(tour))
        return length, tour

    def limits(self):
        tmin = C.c_float()
        tmax = C.c_float()
        lib().orc_colony_limits(self._h, C.byref(tmin), C.byref(tmax))
        return np.float32(tmin.value), np.float32(tmax.value)

    def state(self):
        n = self.n
        d = np.zeros((n, n), np.int32)
        eb = np.zeros((n, n), np.float32)
        cand = np.zeros((n, max(self.cl, 1)), np.int32)
        tau = np.zeros((n, n), np.float32)
        ch = np.zeros((n, n), np.float32)
        lib().orc_colony_get(self._h, _i32p(d), _f32p(eb), _i32p(cand), _f32p(tau), _f32p(ch))
        return {"d": d, "eta_beta": eb, "cand": cand[:, :self.cl], "tau": tau, "choice": ch}

    def tours(self):
        tours = np.zeros((self.m, self.n), np.int32)
        lens = np.zeros(self.m, np.int64)
        fb = np.zeros(self.m, np.int64)
        lib().orc_colony_tours(self._h, _i32p(tours), _i64p(lens), _i64p(fb))
        return tours, lens, fb

    def construct(self, it: int, ant: int):
        """Tour of one ant at iteration ``it`` under the current pheromone."""
        tour = np.zeros(self.n, np.int32)
        fb = C.c_int64()
        length = lib().orc_colony_construct(self._h, it, ant, _i32p(tour), C.byref(fb))
        return length, tour, fb.value

    def step_keys(self, it, ant, t, i, visited):
        """Keys of the competing nodes at one step; (mode, keys) as in orc_step_keys."""
        vis = np.ascontiguousarray(visited, dtype=np.uint8)
        keys = np.zeros(self.n, np.float64)
        mode = lib().orc_step_keys(self._h, it, ant, t, i,
                                   vis.ctypes.data_as(C.POINTER(C.c_uint8)), _f64p(keys))
        return mode, keys

    def variant_step(self, it, ant, prefix, t):
        """Step t of a whole-row variant replayed on prefix[0..t) (orc_variant_step).

        Returns (pick, order, val, u): the oracle's node, the selectable
        positions' nodes, what the selection compares at each position
        (weights for the roulette wheel, keys for reservoir sampling) and the
        roulette wheel's draw."""
        pre = np.ascontiguousarray(prefix[:t], dtype=np.int32)
        order = np.zeros(self.n, np.int32)
        val = np.zeros(self.n, np.float64)
        npos = C.c_int32()
        u = C.c_double()
        pick = lib().orc_variant_step(self._h, it, ant, _i32p(pre), t, _i32p(order), _f64p(val),
                                      C.byref(npos), C.byref(u))
        k = npos.value
        return pick, order[:k], val[:k], u.value
