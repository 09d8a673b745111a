"""Benchmark of the MMAS hot path on GB300 (one JSON line on stdout).

A step is one MMAS iteration (Alg. 1's main loop body): construction by m ants
with candidate lists, bitmask tabu and reservoir sampling, tour lengths,
iteration/global best and limits, and the fused evaporation + deposit +
choice_info pass.  The default workload is the n = 1000 uniform instance,
m = 1000 ants, 32-nearest-neighbour candidate lists, rho = 0.02, alpha = 1,
beta = 2, p_best = 0.01 (synthetic coordinates, seed 1001).

  value        tours/s over K device-timed steps (CUDA events inside the
               iteration graph, on the launching stream), inputs resident in
               HBM, L2 flushed (256 MiB write) before every step;
  e2e          the same metric through the public C ABI with host buffers:
               mmas_create from host coordinates, then per step mmas_iterate
               and mmas_best_tour into host memory;
  roofline     the construction kernel (the dominant one): logical bytes per
               launch (8 cl bytes a step: each candidate's 4-byte weight and
               4-byte id) / its mean CUDA-event duration, against the measured
               HBM copy bandwidth; roofline_l2 the same against the L2 read
               bandwidth measured in the run, roofline_alu against the draw
               rate (the bytes come from shared memory and L2, and the
               step-to-step chain binds);
  cpu_baseline the CPU oracle (test infrastructure) on the host cores, a
               bounded sample of the same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 run under torch.distributed.run; every rank runs an independent
colony (seed + rank) on its own GPU and rank 0 prints the line (weak scaling,
no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

_PRIOR_TRAIN = dict(train_count=2000, train_seed=2000, train_iters=30, train_steps=8, lr=2e-3)
WORKLOADS = {
    # name: (n, m, cl, instance kind, instance seed)
    "uniform-n1000-cl32": dict(n=1000, m=1000, cl=32, kind="uniform", iseed=1001),
    "uniform-n200-fullrow": dict(n=200, m=200, cl=0, kind="uniform", iseed=1002),
    # the same whole-row workload under the paper's other selection / tabu variants
    "uniform-n200-fullrow-rwm": dict(n=200, m=200, cl=0, kind="uniform", iseed=1002, selection=1),
    "uniform-n200-fullrow-rwm-ct": dict(n=200, m=200, cl=0, kind="uniform", iseed=1002, selection=1,
                                        tabu=1),
    "uniform-n200-fullrow-ct": dict(n=200, m=200, cl=0, kind="uniform", iseed=1002, tabu=1),
    "clustered-n3800-cl16-2opt": dict(n=3800, m=1000, cl=16, kind="clustered", iseed=1003, ls=1),
    # plain MMAS on the learned-prior race instances (m = n, cl = 16, no local search): the
    # construction at large n
    "uniform-n5000-cl16": dict(n=5000, m=5000, cl=16, kind="uniform", iseed=1005),
    "uniform-n18500-cl16": dict(n=18500, m=18500, cl=16, kind="uniform", iseed=1018),
    # the same construction form as n = 18,500 (32 warps a CTA, nothing staged) at a size whose
    # matrices (4 x 0.4 GB) a full ncu capture can save and restore
    "uniform-n10000-cl16": dict(n=10000, m=10000, cl=16, kind="uniform", iseed=1010),
    # 256 uniform instances, n = round(exp(U[ln 100, ln 2000])) (size seed 1000), coordinate
    # seed 1000 + i, m = n each
    "batched-256-n100-2000-cl32": dict(kind="batched", count=256, lo=100, hi=2000, cl=32,
                                       size_seed=1000),
    # the learned edge prior: trained on elite tours of generated instances (n log-uniform in
    # [200, 2000], size seed 2000, coordinate seeds 5000 + i; each instance's colony run in
    # batches of 256 for train_iters iterations gives its elite tour), then plain and prior
    # MMAS (m = n, cl = 16, 2-opt of the iteration best) raced for equal wall time on a uniform
    # instance of n = 1000, 5000 or 18500
    "learned-prior-n1000-cl16-2opt": dict(kind="prior", n=1000, m=1000, cl=16, iseed=1001, ls=1,
                                          **_PRIOR_TRAIN, race_s=2.0),
    "learned-prior-n5000-cl16-2opt": dict(kind="prior", n=5000, m=5000, cl=16, iseed=1005, ls=1,
                                          **_PRIOR_TRAIN, race_s=6.0),
    "learned-prior-n18500-cl16-2opt": dict(kind="prior", n=18500, m=18500, cl=16, iseed=1018, ls=1,
                                           **_PRIOR_TRAIN, race_s=15.0),
}
DEFAULT_STEPS = {"uniform-n1000-cl32": 1000, "uniform-n200-fullrow": 1000,
                 "uniform-n200-fullrow-rwm": 1000, "uniform-n200-fullrow-rwm-ct": 1000,
                 "uniform-n200-fullrow-ct": 1000,
                 "clustered-n3800-cl16-2opt": 100, "batched-256-n100-2000-cl32": 30,
                 "uniform-n5000-cl16": 100, "uniform-n18500-cl16": 20, "uniform-n10000-cl16": 50,
                 "learned-prior-n1000-cl16-2opt": 200, "learned-prior-n5000-cl16-2opt": 30,
                 "learned-prior-n18500-cl16-2opt": 10}
PARAMS = dict(alpha=1.0, beta=2.0, rho=0.02, p_best=0.01)
# kernels in one iteration graph: construct, score, update; with 2-opt of the
# iteration best also the 2-opt and the best/limits kernel; with 2-opt of every
# ant the 2-opt kernel before scoring
KERNELS_PER_ITERATION = {0: 3, 1: 5, 2: 4}
METRIC = "candidate tours/sec (one MMAS iteration per step)"
UNIT = "tours/s"
FLUSH_BYTES = 256 << 20
CONSTRUCT_SOURCES = ["paper_2003_11902_gb300/csrc/construct.cu",
                     "paper_2003_11902_gb300/csrc/internal.cuh"]


def _instance(w):
    from paper_2003_11902_gb300 import instances as I
    if w["kind"] in ("uniform", "prior"):
        return I.uniform(w["n"], w["iseed"])
    return I.clustered(w["n"], w["iseed"])


def _batch_instances(w):
    from paper_2003_11902_gb300 import instances as I
    ns = I.log_uniform_sizes(w["count"], w["size_seed"], w["lo"], w["hi"])
    return [I.uniform(int(n), 1000 + i) for i, n in enumerate(ns)]


def _batch_cfg(w, xys):
    ns = [len(x) for x in xys]
    return {"colonies": w["count"], "n": f"log-uniform [{w['lo']}, {w['hi']}]", "n_min": min(ns),
            "n_max": max(ns), "total_ants": sum(ns), "m": "n per colony", "cl": w["cl"],
            "instance": "uniform, size seed 1000, coordinate seed 1000 + i", **PARAMS}


def _variant(w):
    """Whole-row selection / tabu variant of a workload (both 0 by default)."""
    return {"selection": w.get("selection", 0), "tabu": w.get("tabu", 0)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _source_sha(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _profiled_traffic(workload):
    """DRAM bytes per construction launch from the committed ncu summary, if the
    kernel source is unchanged since the capture; else None."""
    path = os.path.join(ROOT, "profiles", f"construct_{workload}.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("source_sha") != _source_sha(CONSTRUCT_SOURCES):
        return None
    return rec.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mmas_clocks_{os.getpid()}.csv")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={device_index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(w, xy, budget_s=12.0):
    """The oracle as it stands, all host cores, whole iterations until budget_s."""
    import oracle as O
    cores = os.cpu_count() or 1
    col = O.Colony(xy=xy, m=w["m"], cl=w["cl"], seed=1, ls=w.get("ls", 0), **_variant(w), **PARAMS)
    it, t0 = 0, time.perf_counter()
    while True:
        col.iterate(1, threads=cores)
        it += 1
        el = time.perf_counter() - t0
        if el >= budget_s or it >= 200:
            break
    return {"value": w["m"] * it / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{it} whole iterations (all {w['m']} ants + pheromone update) of the "
                      f"same workload, OpenMP over ants on {cores} threads, {el:.1f} s"}


def cpu_baseline_sample(w, xy, budget_s=12.0):
    """The oracle as it stands, all host cores, for instances whose whole
    iterations outlast the budget: ants of one iteration constructed in parallel
    until budget_s (set-up untimed)."""
    import concurrent.futures as cf

    import oracle as O
    cores = os.cpu_count() or 1
    col = O.Colony(xy=xy, m=w["m"], cl=w["cl"], seed=1, **PARAMS)
    it, done, t0 = col.iteration, 0, time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        while done < w["m"]:
            ants = range(done, min(done + cores, w["m"]))
            list(ex.map(lambda k: col.construct(it, int(k)), ants))
            done += len(ants)
            if time.perf_counter() - t0 >= budget_s:
                break
    el = time.perf_counter() - t0
    return {"value": done / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} of {w['m']} ants of one iteration constructed (construction only: no "
                      f"local search or pheromone update; set-up untimed), {cores} threads, {el:.1f} s"}


def run_reference(args, w):
    """--impl reference: the CPU oracle times the same workload on the host cores."""
    ws, rank, _ = _dist_env()
    if rank != 0:
        return
    import oracle as O
    xy = _instance(w)
    cores = os.cpu_count() or 1
    col = O.Colony(xy=xy, m=w["m"], cl=w["cl"], seed=1, ls=w.get("ls", 0), **_variant(w), **PARAMS)
    t0 = time.perf_counter()
    col.iterate(1, threads=cores)
    t_iter = time.perf_counter() - t0
    budget = 150.0
    full = (args.steps + args.warmup) * t_iter <= budget
    if full:
        for _ in range(max(0, args.warmup - 1)):
            col.iterate(1, threads=cores)
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            col.iterate(1, threads=cores)
            times.append(time.perf_counter() - t0)
        tours = w["m"] * args.steps
        sample = f"whole iterations ({w['m']} ants + pheromone update), {cores} threads"
    else:
        # bounded sample: each step constructs S ants of the current iteration
        import concurrent.futures as cf
        s_ants = max(cores, int(w["m"] * budget / ((args.steps + args.warmup) * t_iter)))
        s_ants = min(s_ants, w["m"])
        it = col.iteration
        ants = np.linspace(0, w["m"] - 1, s_ants).astype(int)
        times = []
        with cf.ThreadPoolExecutor(max_workers=cores) as ex:
            for step in range(args.warmup + args.steps):
                t0 = time.perf_counter()
                list(ex.map(lambda k: col.construct(it, int(k)), ants))
                if step >= args.warmup:
                    times.append(time.perf_counter() - t0)
        tours = s_ants * args.steps
        sample = (f"{s_ants} of {w['m']} ants constructed per step (construction only), "
                  f"{cores} threads")
    total = sum(times)
    value = tours / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, **_cfg(w)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _cfg(w):
    kind = "uniform" if w["kind"] == "prior" else w["kind"]  # the prior races on uniform instances
    c = {"n": w["n"], "m": w["m"], "cl": w["cl"], "instance": f"{kind} seed {w['iseed']}",
         **PARAMS}
    if w.get("ls"):
        c["local_search"] = "2-opt of the iteration best" if w["ls"] == 1 else "2-opt of every ant"
    if w.get("cl") == 0:
        c["selection"] = "roulette wheel" if w.get("selection") else "weighted reservoir sampling"
        c["tabu"] = "compact list" if w.get("tabu") else "bitmask"
    return c


def algorithmic_construct_bytes(w):
    """Logical bytes a construction launch reads, counted as the method's unit
    of work: per step, each of the cl candidates' weight (4 B) and id (4 B) --
    8 cl bytes a step, 256 B at cl = 32 -- or, without candidate lists, the
    weight (4 B) of each of the n - t unvisited nodes at step t."""
    n, m, cl = w["n"], w["m"], w["cl"]
    if cl > 0:
        per_ant = (n - 1) * cl * 8
    else:
        per_ant = 4 * (n * (n - 1) // 2)
    return m * per_ant


def stored_construct_bytes(w):
    """The same reads as this library stores them: 16-bit candidate ids (2 B)
    and reciprocal weights (4 B) per candidate and step, plus the 4-byte tour
    entry per step (whole rows: the unvisited weights and the tour entries)."""
    n, m, cl = w["n"], w["m"], w["cl"]
    if cl > 0:
        per_ant = (n - 1) * cl * 6 + 4 * n
    else:
        per_ant = 4 * (n * (n - 1) // 2) + 4 * n
    return m * per_ant


def memory_rooflines(w, c_ms, dev, traffic=None):
    """The construction kernel's logical bytes per second against the measured
    HBM copy peak and against the L2 read bandwidth measured in this run
    (mmas_probe_l2_bandwidth over a 32 MiB L2-resident buffer)."""
    from paper_2003_11902_gb300 import mmas as _mm
    peak, peak_kind = _peaks()
    algo = algorithmic_construct_bytes(w)
    achieved = algo / (c_ms * 1e-3) / 1e9
    l2 = _mm.mmas_probe_l2_bandwidth(dev, 32 << 20)
    hbm = {"kernel": "k_construct", "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
           "algorithmic_bytes_per_launch": algo,
           "bytes_per_step": algo / (w["m"] * (w["n"] - 1)),
           "stored_bytes_per_launch": stored_construct_bytes(w),
           "stored_frac": stored_construct_bytes(w) / (c_ms * 1e-3) / 1e9 / peak}
    l2line = {"kernel": "k_construct", "bound": "l2", "achieved": achieved, "peak": l2, "unit": "GB/s",
              "frac": achieved / l2,
              "peak_kind": "measured (mmas_probe_l2_bandwidth: 16-byte L2-only loads over a 32 MiB "
                           "resident buffer, best of 10, same run)"}
    return hbm, l2line


# L* of a workload: the oracle's long-run best (tests/golden/make_lstar.py)
LSTAR_FILES = {"uniform-n1000-cl32": ("lstar_uniform_n1000.json", "seeds 1-3, 1000 iterations"),
               "clustered-n3800-cl16-2opt": ("lstar_clustered_n3800.json",
                                             "seeds 1-3, 500 iterations with 2-opt of the iteration best"),
               "learned-prior-n1000-cl16-2opt": ("lstar_uniform_n1000_cl16_2opt.json",
                                                 "plain MMAS, seeds 1-3, 1000 iterations with 2-opt of the "
                                                 "iteration best")}


def time_to_gap(workload, w, xy, seed, dev, stream, gap=0.02, check_every=5, max_iters=4000):
    """Wall time from mmas_create until the colony's global best is within `gap`
    of the oracle's long-run best L* (tests/golden), checking every few
    iterations (each check reads the best length back to the host)."""
    from paper_2003_11902_gb300 import Colony
    if workload not in LSTAR_FILES:
        return None
    fname, how = LSTAR_FILES[workload]
    path = os.path.join(ROOT, "tests", "golden", fname)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        lstar = json.load(f)["lstar"]
    target = (1.0 + gap) * lstar
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    col = Colony(xy=xy, m=w["m"], cl=w["cl"], seed=seed, ls=w.get("ls", 0), device=dev, stream=stream,
                 **PARAMS)
    it, best = 0, None
    while it < max_iters:
        col.iterate(check_every)
        it += check_every
        best = col.stats()["best_len"]
        if best <= target:
            break
    el = time.perf_counter() - t0
    col.close()
    return {"seconds": el if best <= target else None, "iterations": it, "best_len": best,
            "lstar": lstar, "target": target, "seed": seed,
            "timed": f"mmas_create + iterations + a best-length read every {check_every} iterations",
            "lstar_source": f"tests/golden/{fname} (oracle, {how})"}


def run_ours(args, w):
    import torch
    import torch.distributed as dist

    from paper_2003_11902_gb300 import Colony, _build, mmas

    ws, rank, local = _dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.cuda.current_device()
    _build.build()
    xy = _instance(w)
    seed = 1 + rank
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)  # the flush, the colony and all timing share this stream
    col = Colony(xy=xy, m=w["m"], cl=w["cl"], seed=seed, device=dev, ls=w.get("ls", 0),
                 stream=stream.cuda_stream, **_variant(w), **PARAMS)
    col.enable_phase_timing(True)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        col.iterate(1)
    col.synchronize()

    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev) if rank == 0 else None
    con, tot = [], []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        col.iterate(1)
        c, _, t = col.phase_times()  # synchronises the stream
        con.append(c)
        tot.append(t)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop() if sampler else None
    if ws > 1:
        dist.barrier()
    total_ms = float(sum(tot))
    if ws > 1:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    st = col.stats()
    best_len, _ = col.best_tour()

    # end to end through the C ABI with host buffers
    e2e_total = 0.0
    t0 = time.perf_counter()
    col2 = Colony(xy=xy, m=w["m"], cl=w["cl"], seed=seed, device=dev, ls=w.get("ls", 0),
                  stream=stream.cuda_stream, **_variant(w), **PARAMS)
    col2.synchronize()
    e2e_total += time.perf_counter() - t0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        col2.iterate(1)
        col2.best_tour()  # device -> host: scalar block + best tour
        e2e_total += time.perf_counter() - t0
    col2.close()
    e2e_value = w["m"] * args.steps / e2e_total
    if ws > 1:
        t = torch.tensor([e2e_total], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_value = ws * w["m"] * args.steps / float(t.item())

    if rank == 0:
        c_ms = statistics.mean(con)
        roof, roof_l2 = memory_rooflines(w, c_ms, dev, _profiled_traffic(args.workload))
        value = ws * w["m"] * args.steps / (total_ms * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, **_cfg(w), "parallelism": f"replicas{ws}",
                       "l2": "flushed before every step (256 MiB write)",
                       "timing": "CUDA events in the iteration graph, launching stream"},
            "construct_ms": c_ms,
            "after_construct_ms": statistics.mean(t - c for t, c in zip(tot, con)),
            "construct_tours_per_s": w["m"] / (c_ms * 1e-3),
            "roofline": roof,
            "roofline_l2": roof_l2,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * w["n"] / args.steps,
                    "d2h_bytes_per_step": 4 * w["n"] + 64},
            "gpu_launches": KERNELS_PER_ITERATION[w.get("ls", 0)] * args.steps,
            "clocks": clocks,
            "best_len": best_len, "fallback_steps": st["fallback_steps"],
            "wall_s": wall,
            "paper_context": "V100, pr1002, cl=32, MMAS-WRS-BT: 0.93 ms construction "
                             "(~1.08M tours/s), Table 6",
        }
        if w["cl"] > 0:
            # the same kernel against the arithmetic ceiling of its steps: every
            # candidate slot draws at every step (Philox word, log2, key), measured
            # at full occupancy by the library's probe in this run
            from paper_2003_11902_gb300 import mmas as _mm
            draws = w["m"] * (w["n"] - 1) * w["cl"]
            rate = _mm.mmas_probe_draw_rate(dev, 50.0) / 1e9
            sched = 4 * torch.cuda.get_device_properties(dev).multi_processor_count
            got = draws / (c_ms * 1e-3) / 1e9
            line["roofline_alu"] = {
                "kernel": "k_construct", "bound": "alu", "achieved": got, "peak": rate,
                "unit": "Gdraws/s", "frac": got / rate, "algorithmic_draws_per_launch": draws,
                "peak_kind": "measured (mmas_probe_draw_rate: Philox + log2 + key per draw at full "
                             "occupancy, same run)",
                "binding": f"neither: the step-to-step dependency chain of each ant (about 300 "
                           f"cycles a step) with {w['m']} ants on {sched} warp schedulers"}
        gapres = None if args.no_gap else time_to_gap(args.workload, w, xy, seed, dev, stream.cuda_stream)
        if gapres is not None:
            line["time_to_2pct_gap"] = gapres
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = (cpu_baseline if w["n"] <= 2000 else cpu_baseline_sample)(w, xy)
        print(json.dumps(line), flush=True)
    col.close()
    if ws > 1:
        dist.destroy_process_group()


def cpu_baseline_batch(w, xys, budget_s=12.0):
    """The oracle as it stands, all host cores: one whole iteration of each colony
    in turn, from the first, until budget_s."""
    import oracle as O
    cores = os.cpu_count() or 1
    tours, done, el = 0, 0, 0.0
    for b, xy in enumerate(xys):
        col = O.Colony(xy=xy, m=len(xy), cl=w["cl"], seed=1 + b, **PARAMS)  # set-up, untimed
        t0 = time.perf_counter()
        col.iterate(1, threads=cores)
        el += time.perf_counter() - t0
        tours += len(xy)
        done += 1
        if el >= budget_s:
            break
    return {"value": tours / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one whole iteration of each of the first {done} of {len(xys)} colonies "
                      f"({tours} ants; set-up untimed), OpenMP over ants on {cores} threads, "
                      f"{el:.1f} s"}


def run_reference_batch(args, w):
    ws, rank, _ = _dist_env()
    if rank != 0:
        return
    xys = _batch_instances(w)
    cores = os.cpu_count() or 1
    import oracle as O
    # each step: whole iterations of colonies taken in turn, bounded to ~budget / steps
    per_step = 150.0 / (args.steps + args.warmup)
    cols = {}
    nxt = 0
    times, tours = [], 0
    for step in range(args.warmup + args.steps):
        el, done = 0.0, 0
        while el < per_step:
            b = nxt % len(xys)
            nxt += 1
            if b not in cols:  # set-up, untimed
                cols[b] = O.Colony(xy=xys[b], m=len(xys[b]), cl=w["cl"], seed=1 + b, **PARAMS)
            t0 = time.perf_counter()
            cols[b].iterate(1, threads=cores)
            el += time.perf_counter() - t0
            done += len(xys[b])
        if step >= args.warmup:
            times.append(el)
            tours += done
    total = sum(times)
    value = tours / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, **_batch_cfg(w, xys)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"whole colony iterations taken in turn, ~{per_step:.1f} s "
                                       f"per step (set-up untimed), {cores} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours_batch(args, w):
    import torch
    import torch.distributed as dist

    from paper_2003_11902_gb300 import Batch, _build, mmas

    ws, rank, local = _dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.cuda.current_device()
    _build.build()
    xys = _batch_instances(w)
    ns = [len(x) for x in xys]
    total_ants = sum(ns)
    seed = 1 + rank * w["count"]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    bt = Batch(xys=xys, m=0, cl=w["cl"], seed=seed, device=dev, stream=stream.cuda_stream,
               **PARAMS)
    tuned = bt.autotune(reps=3)
    bt.enable_phase_timing(True)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        bt.iterate(1)
    bt.synchronize()
    fb0 = bt.fallback_steps()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev) if rank == 0 else None
    con, tot = [], []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        bt.iterate(1)
        c, _, t = bt.phase_times()
        con.append(c)
        tot.append(t)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop() if sampler else None
    fb = bt.fallback_steps() - fb0
    if ws > 1:
        dist.barrier()
    total_ms = float(sum(tot))
    if ws > 1:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    best = bt.best_lengths()

    # end to end through the C ABI with host buffers: create from host
    # coordinates, then per step iterate and read every colony's best length
    e2e_total = 0.0
    t0 = time.perf_counter()
    bt2 = Batch(xys=xys, m=0, cl=w["cl"], seed=seed, device=dev, stream=stream.cuda_stream,
                **PARAMS)
    bt2.set_config(*tuned)
    bt2.synchronize()
    e2e_total += time.perf_counter() - t0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bt2.iterate(1)
        bt2.best_lengths()
        e2e_total += time.perf_counter() - t0
    bt2.close()
    e2e_value = total_ants * args.steps / e2e_total

    if rank == 0:
        c_ms = statistics.mean(con)
        draws = sum(n * (n - 1) for n in ns) * w["cl"]  # every candidate slot draws each step
        achieved = draws / (c_ms * 1e-3)
        peak = mmas.mmas_probe_draw_rate(dev, 50.0)
        value = ws * total_ants * args.steps / (total_ms * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, **_batch_cfg(w, xys),
                       "parallelism": f"replicas{ws}", "launch_shape": list(tuned),
                       "l2": "flushed before every step (256 MiB write)",
                       "timing": "CUDA events in the iteration graph, launching stream"},
            "construct_ms": c_ms,
            "after_construct_ms": statistics.mean(t - c for t, c in zip(tot, con)),
            "construct_steps_per_s": sum(n * (n - 1) for n in ns) / (c_ms * 1e-3),
            "roofline": {"kernel": "k_construct_batch", "bound": "alu", "achieved": achieved / 1e9,
                         "peak": peak / 1e9, "unit": "Gdraws/s", "frac": achieved / peak,
                         "peak_kind": "measured (mmas_probe_draw_rate: Philox + log2 + key per "
                                      "draw at full occupancy, same run)",
                         "traffic": None, "algorithmic_draws_per_launch": draws},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 4 * w["count"],
                    "note": "create from host coordinates + per step iterate and read all best lengths"},
            "gpu_launches": 3 * args.steps,
            "clocks": clocks,
            "best_len_mean": float(np.mean(best)), "fallback_steps": int(fb),
            "wall_s": wall,
        }
        if ws == 1:
            line["vs_single_colonies"] = _single_colonies(w, xys, seed, dev, stream.cuda_stream,
                                                          args.warmup + args.steps, args.steps,
                                                          total_ms, best)
            if not args.no_gap:
                line["time_to_2pct_gap"] = batch_time_to_gap(w, seed, dev, stream.cuda_stream)
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_batch(w, xys)
        print(json.dumps(line), flush=True)
    bt.close()
    if ws > 1:
        dist.destroy_process_group()


def _single_colonies(w, xys, seed, dev, stream, iters, timed, batch_ms, batch_best):
    """The batch's colonies run one at a time as ordinary colonies (colony b with
    seed + b), for the same iterations: device time of the last `timed`
    iterations of each, summed, against the batch's; and whether every colony
    reaches the same best length (the batch equals its colonies run alone)."""
    from paper_2003_11902_gb300 import Colony

    ms, same = 0.0, True
    for b, xy in enumerate(xys):
        col = Colony(xy=xy, m=len(xy), cl=w["cl"], seed=seed + b, device=dev, stream=stream, **PARAMS)
        col.iterate(iters - timed)
        col.enable_phase_timing(True)
        for _ in range(timed):
            col.iterate(1)
            ms += col.phase_times()[2]
        same = same and col.best_tour()[0] == int(batch_best[b])
        col.close()
    return {"colonies": len(xys), "iterations_each": iters, "timed_iterations": timed,
            "single_ms_per_iteration_of_all": ms / timed, "batched_ms_per_iteration": batch_ms / timed,
            "speedup": ms / batch_ms, "same_best_lengths": bool(same),
            "note": "device time (CUDA events in each colony's iteration graph); the batch and the "
                    "colonies run alone build the same tours, so any time-to-quality ratio is this one"}


def batch_time_to_gap(w, seed, dev, stream, gap=0.02, check_every=5, max_iters=4000):
    """Wall time for the sampled instances of the batched workload (the oracle's
    L* of each in tests/golden/lstar_batched_sample16.json) to come within `gap`
    of their L*: as one batch (create, then iterate; the time at which each
    colony first is within), and as plain colonies run one after another
    (create, then iterate until within).  Colony b gets seed + b either way, so
    both build the same tours and the same colonies reach the target within
    `max_iters`; over those, the batch's time is the last one to reach it and
    the plain colonies' time is the sum of theirs.  Every check reads the best
    lengths back."""
    import torch

    from paper_2003_11902_gb300 import Batch, Colony
    from paper_2003_11902_gb300 import instances as I
    path = os.path.join(ROOT, "tests", "golden", "lstar_batched_sample16.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        insts = json.load(f)["instances"]
    xys = [I.uniform(e["n"], 1000 + e["index"]) for e in insts]
    target = np.array([(1.0 + gap) * e["lstar"] for e in insts])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bt = Batch(xys=xys, m=0, cl=w["cl"], seed=seed, device=dev, stream=stream, **PARAMS)
    hit_s = [None] * len(xys)
    hit_it = [None] * len(xys)
    it = 0
    while it < max_iters and None in hit_s:
        bt.iterate(check_every)
        it += check_every
        best = bt.best_lengths()
        el = time.perf_counter() - t0
        for b in range(len(xys)):
            if hit_s[b] is None and best[b] <= target[b]:
                hit_s[b], hit_it[b] = el, it
    bt.close()
    single_s, single_it = 0.0, []
    for b, xy in enumerate(xys):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        col = Colony(xy=xy, m=len(xy), cl=w["cl"], seed=seed + b, device=dev, stream=stream, **PARAMS)
        k, ok = 0, False
        while k < max_iters and not ok:
            col.iterate(check_every)
            k += check_every
            ok = col.stats()["best_len"] <= target[b]
        el = time.perf_counter() - t0
        col.close()
        single_it.append(k if ok else None)
        if ok:
            single_s += el
    reached = [b for b in range(len(xys)) if hit_s[b] is not None]
    batch_s = max(hit_s[b] for b in reached) if reached else None
    return {"instances": [[e["index"], e["n"]] for e in insts], "max_iterations": max_iters,
            "reached": len(reached), "batch_seconds": batch_s, "batch_iterations": hit_it,
            "single_seconds_total": single_s if reached else None, "single_iterations": single_it,
            "same_iterations": hit_it == single_it,
            "speedup": single_s / batch_s if batch_s else None,
            "timed": f"create + iterations + a best-length read every {check_every} iterations; "
                     "times over the colonies that reach the target",
            "lstar_source": "tests/golden/lstar_batched_sample16.json (oracle, per instance the best of "
                            "seeds 1-3, 1000 iterations)"}


def _race(col, seconds, target, check_every=5):
    """Iterate until `seconds` of wall time; the best length after each check
    and the time at which it first reached `target`."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    trace, hit = [], None
    while True:
        col.iterate(check_every)
        best = col.stats()["best_len"]
        el = time.perf_counter() - t0
        trace.append((round(el, 4), int(best)))
        if hit is None and best <= target:
            hit = el
        if el >= seconds:
            break
    return trace, hit


def _race_from_create(make, seconds, check_every=5):
    """Wall-clock race of one colony, the clock started before make() (which
    creates the colony and applies whatever heuristic it uses): the best length
    after every check, with the time since the start.  Returns the trace, the
    colony and the seconds make() took."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    col = make()
    col.synchronize()
    setup_s = time.perf_counter() - t0
    trace = []
    while True:
        col.iterate(check_every)
        best = col.stats()["best_len"]
        el = time.perf_counter() - t0
        trace.append((round(el, 4), int(best)))
        if el >= seconds:
            break
    return trace, col, setup_s


def _train_prior(prior, w, count, dev, stream):
    """Train `prior` on the elite tours of `count` generated instances: each
    chunk of 256 runs as one batch of colonies (m = n) for train_iters
    iterations, then every colony's best tour, improved by the colony's 2-opt
    (mmas_two_opt_tour, as the races' colonies apply it), drives train_steps
    Adam steps on that colony.  Returns the wall time and the mean first / last loss per chunk."""
    from paper_2003_11902_gb300 import Batch
    from paper_2003_11902_gb300 import instances as I

    sizes = I.log_uniform_sizes(count, w["train_seed"], 200, 2000)
    t0 = time.perf_counter()
    by_chunk = []
    for c0 in range(0, count, 256):
        xys = [I.uniform(int(n), 5000 + c0 + i) for i, n in enumerate(sizes[c0:c0 + 256])]
        bt = Batch(xys=xys, m=0, cl=w["cl"], seed=100 + c0, device=dev, stream=stream, **PARAMS)
        bt.iterate(w["train_iters"])
        first, last = [], []
        for c in range(len(xys)):
            _, elite = bt.best_tour(c)
            col = bt.colony(c)
            elite, _ = col.two_opt(elite)  # improved by 2-opt, as the races' colonies improve theirs
            first.append(prior.train(col, elite, steps=1, lr=w["lr"]))
            last.append(prior.train(col, elite, steps=w["train_steps"] - 1, lr=w["lr"]))
            col.close()
        bt.close()
        by_chunk.append((round(float(np.mean(first)), 4), round(float(np.mean(last)), 4)))
    return time.perf_counter() - t0, sizes, by_chunk


def _break_even(race, train_s):
    """How many evaluated instances like this one amortise the one-off training:
    train_s / (time the plain colony needs to the target - the prior's), per
    prior form; None when the prior is not faster or a colony misses."""
    out = {}
    tp = race["plain"].get("seconds_to_target")
    for name in ("prior", "prior_weighted"):
        t = race[name].get("seconds_to_target")
        out[name] = (round(train_s / (tp - t), 1) if tp is not None and t is not None and tp > t else None)
    return out


def run_ours_prior(args, w):
    import torch

    from paper_2003_11902_gb300 import Colony, Prior, _build
    from paper_2003_11902_gb300 import instances as I

    _, rank, _ = _dist_env()
    dev = torch.cuda.current_device()
    _build.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    common = dict(cl=w["cl"], device=dev, ls=w["ls"], stream=stream.cuda_stream, **PARAMS)
    # ---- training on elite tours of generated instances
    prior = Prior(I.prior_params(1), device=dev)
    count = args.train_instances or w["train_count"]
    train_s, sizes, by_chunk = _train_prior(prior, w, count, dev, stream.cuda_stream)
    # ---- equal-wall-time race on the evaluation instance
    xy = _instance(w)
    lstar = None
    if args.workload in LSTAR_FILES:
        fname, how = LSTAR_FILES[args.workload]
        path = os.path.join(ROOT, "tests", "golden", fname)
        if os.path.exists(path):
            with open(path) as f:
                lstar = json.load(f)["lstar"]
    # three colonies: plain eta^beta, eta^beta replaced by the edge
    # probabilities, and eta^beta weighted by them (gamma = 1).  Each race's
    # clock starts before mmas_create and includes applying the prior, so the
    # three times to the target are measured the same way; the training is a
    # one-off cost reported beside them.
    def make_plain():
        return Colony(xy=xy, m=w["m"], seed=1, **common)

    def make_replaced():
        col = Colony(xy=xy, m=w["m"], seed=1, **common)
        prior.apply(col)
        return col

    def make_weighted():
        col = Colony(xy=xy, m=w["m"], seed=1, **common)
        prior.apply_weighted(col, 1.0)
        return col

    race = {}
    for name, make in (("plain", make_plain), ("prior", make_replaced), ("prior_weighted", make_weighted)):
        trace, col, setup_s = _race_from_create(make, w["race_s"])
        race[name] = {"best_at_end": trace[-1][1], "trace": trace, "create_and_apply_s": round(setup_s, 4)}
        if name == "prior":
            guided = col
        else:
            col.close()
    apply_s = race["prior"]["create_and_apply_s"]
    # the time each colony first came within 2% of the target: L* (the
    # oracle's long-run best) where it is known, else the best final length
    # of the three colonies
    if lstar is not None:
        target, target_source = 1.02 * lstar, f"1.02 L*, L* from tests/golden/{fname} (oracle, {how})"
    else:
        target = 1.02 * min(r["best_at_end"] for r in race.values())
        target_source = ("1.02 x the best final length of the three colonies (no oracle L* at this size): "
                         "time to 2% of the race's best, not of an oracle L*")
    for r in race.values():
        r["seconds_to_target"] = next((t for t, b in r["trace"] if b <= target), None)
        r["trace"] = r["trace"][::max(1, len(r["trace"]) // 40)]
    # ---- throughput of the prior-guided colony (as for the other workloads)
    guided.enable_phase_timing(True)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        guided.iterate(1)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev) if rank == 0 else None
    con, tot = [], []
    for _ in range(args.steps):
        flush.zero_()
        guided.iterate(1)
        c, _, t = guided.phase_times()
        con.append(c)
        tot.append(t)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    total_ms = float(sum(tot))
    # end to end: create from host coordinates, apply the prior, then per step
    # iterate and read the best tour back
    t0 = time.perf_counter()
    e2e_col = Colony(xy=xy, m=w["m"], seed=1, **common)
    prior.apply(e2e_col)
    for _ in range(args.steps):
        e2e_col.iterate(1)
        e2e_col.best_tour()
    e2e_s = time.perf_counter() - t0
    e2e_col.close()
    guided.close()
    prior.close()
    c_ms = statistics.mean(con)
    wc = dict(w, n=w["n"], m=w["m"], cl=w["cl"])
    roof, roof_l2 = memory_rooflines(wc, c_ms, 0)
    line = {
        "metric": METRIC, "value": w["m"] * args.steps / (total_ms * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": w["n"], "m": w["m"], "cl": w["cl"],
                   "instance": f"uniform seed {w['iseed']}", "local_search": "2-opt of the iteration best",
                   "heuristic": "learned edge prior (3-layer message passing, hidden 64, bf16 tensor cores)",
                   **PARAMS, "parallelism": "replicas1",
                   "l2": "flushed before every step (256 MiB write)",
                   "timing": "CUDA events in the iteration graph, launching stream"},
        "construct_ms": c_ms,
        "after_construct_ms": statistics.mean(t - c for t, c in zip(tot, con)),
        "roofline": roof,
        "roofline_l2": roof_l2,
        "e2e": {"value": w["m"] * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 4 * w["n"] + 64,
                "note": "create + apply the trained prior + per step iterate and read the best tour"},
        "gpu_launches": KERNELS_PER_ITERATION[w["ls"]] * args.steps,
        "clocks": clocks,
        "learned_prior": {
            "train_instances": len(sizes), "train_n_range": [int(sizes.min()), int(sizes.max())],
            "train_iters": w["train_iters"], "train_steps": w["train_steps"],
            "train_s": round(train_s, 3), "loss_first_last_per_256": by_chunk,
            "train_s_per_training_instance": round(train_s / len(sizes), 5),
            "apply_s": round(apply_s, 4), "race_seconds": w["race_s"], "target": target,
            "target_source": target_source,
            "clock": "every race from before mmas_create, prior applied inside the clock; "
                     "training (train_s) is a one-off outside it",
            "break_even_evaluations": _break_even(race, train_s),
            "race": race},
    }
    if not args.no_cpu_baseline:
        cb = cpu_baseline if w["n"] <= 2000 else cpu_baseline_sample
        line["cpu_baseline"] = cb(dict(w, m=w["m"]), xy)
        line["cpu_baseline"]["sample"] += " (plain MMAS: the oracle has no learned prior)"
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: the workload's iteration budget, capped)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="uniform-n1000-cl32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-gap", action="store_true", help="skip the time-to-2%%-gap run")
    ap.add_argument("--train-instances", type=int, default=None,
                    help="learned-prior workloads: generated training instances (default 2000)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    w = WORKLOADS[args.workload]
    if args.steps is None:
        args.steps = DEFAULT_STEPS[args.workload]
    if w["kind"] == "batched":
        (run_reference_batch if args.impl == "reference" else run_ours_batch)(args, w)
    elif w["kind"] == "prior" and args.impl != "reference":
        run_ours_prior(args, w)
    elif args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
