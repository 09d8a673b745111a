"""Write the oracle's long-run best tour length L* of a benchmark workload.

L* is the shortest tour the CPU oracle (MMAS, Alg. 1) finds over MMAS seeds
1..3, each run for the workload's full iteration budget, with alpha = 1,
beta = 2, rho = 0.02, p_best = 0.01.  It anchors the time-to-within-2%
measurement.  Calls only the oracle.  Workloads:

  uniform-n1000   synthetic uniform n = 1000 (coordinate seed 1001), m = 1000,
                  cl = 32, 1000 iterations -> lstar_uniform_n1000.json
  uniform-n1000-cl16-2opt  the same instance, m = 1000, cl = 16, 2-opt of each
                  iteration's best, 1000 iterations -> lstar_uniform_n1000_cl16_2opt.json
                  (the plain colony of the learned-prior race at n = 1000)
  clustered-n3800 synthetic clustered n = 3800 (seed 1003), m = 1000, cl = 16,
                  2-opt of each iteration's best (Sec. 5.7), 500 iterations
                  -> lstar_clustered_n3800.json
  uniform-n5000-cl16-2opt  synthetic uniform n = 5000 (coordinate seed 1005),
                  m = 5000, cl = 16, 2-opt of each iteration's best; the plain
                  colony of the learned-prior race at n = 5000.  An oracle
                  iteration there takes tens of seconds on 8 cores, so the
                  default is MMAS seed 1 alone for 200 iterations (stated in
                  the file) -> lstar_uniform_n5000_cl16_2opt.json
  batched-sample16 the first 16 instances with n <= 400 of the batched workload
                  (256 uniform instances, n = round(exp(U[ln 100, ln 2000])) with
                  size seed 1000, coordinate seed 1000 + index), m = n, cl = 32,
                  1000 iterations each -> lstar_batched_sample16.json (one L*
                  per instance; runs go to a pool of single-threaded processes)

    python tests/golden/make_lstar.py [--workload uniform-n1000] [--iters N] [--seeds 1,2,3]
                                      [--threads N]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_2003_11902_gb300 import instances as I  # noqa: E402


WORKLOADS = {
    "uniform-n1000": dict(kind="uniform", n=1000, iseed=1001, m=1000, cl=32, ls=0, iters=1000,
                          out="lstar_uniform_n1000.json",
                          text="uniform n=1000 (coordinate seed 1001), m=1000, cl=32, alpha=1, beta=2, "
                               "rho=0.02, p_best=0.01"),
    "uniform-n1000-cl16-2opt": dict(kind="uniform", n=1000, iseed=1001, m=1000, cl=16, ls=1, iters=1000,
                                    out="lstar_uniform_n1000_cl16_2opt.json",
                                    text="uniform n=1000 (coordinate seed 1001), m=1000, cl=16, 2-opt of the "
                                         "iteration best, alpha=1, beta=2, rho=0.02, p_best=0.01"),
    "clustered-n3800": dict(kind="clustered", n=3800, iseed=1003, m=1000, cl=16, ls=1, iters=500,
                            out="lstar_clustered_n3800.json",
                            text="clustered n=3800 (seed 1003), m=1000, cl=16, 2-opt of the iteration "
                                 "best, alpha=1, beta=2, rho=0.02, p_best=0.01"),
    "uniform-n5000-cl16-2opt": dict(kind="uniform", n=5000, iseed=1005, m=5000, cl=16, ls=1, iters=200,
                                    seeds=(1,), out="lstar_uniform_n5000_cl16_2opt.json",
                                    text="uniform n=5000 (coordinate seed 1005), m=5000, cl=16, 2-opt of the "
                                         "iteration best, alpha=1, beta=2, rho=0.02, p_best=0.01"),
}


def instance(w):
    """The coordinates of a single-colony workload."""
    return I.uniform(w["n"], w["iseed"]) if w["kind"] == "uniform" else I.clustered(w["n"], w["iseed"])


BATCH_SAMPLE = dict(count=256, size_seed=1000, lo=100, hi=2000, max_n=400, take=16, cl=32, iters=1000,
                    out="lstar_batched_sample16.json")


def batch_sample():
    """(index, n) of the sampled instances of the batched workload."""
    b = BATCH_SAMPLE
    ns = I.log_uniform_sizes(b["count"], b["size_seed"], b["lo"], b["hi"])
    return [(i, int(n)) for i, n in enumerate(ns) if n <= b["max_n"]][:b["take"]]


def _run_one(job):
    idx, n, seed, iters = job
    xy = I.uniform(n, 1000 + idx)
    t0 = time.time()
    col = O.Colony(xy=xy, m=n, cl=BATCH_SAMPLE["cl"], alpha=1.0, beta=2.0, rho=float(np.float32(0.02)),
                   p_best=float(np.float32(0.01)), seed=seed)
    col.iterate(iters, threads=1)
    return idx, seed, int(col.best()[0]), round(time.time() - t0, 1)


def main_batch(iters, procs):
    jobs = [(i, n, seed, iters) for i, n in batch_sample() for seed in (1, 2, 3)]
    jobs.sort(key=lambda j: -j[1])  # largest first
    with mp.get_context("spawn").Pool(procs) as pool:
        res = list(pool.imap_unordered(_run_one, jobs))
    insts = []
    for i, n in batch_sample():
        runs = sorted((r for r in res if r[0] == i), key=lambda r: r[1])
        insts.append({"index": i, "n": n, "lstar": min(r[2] for r in runs),
                      "runs": [{"seed": r[1], "best": r[2], "seconds": r[3]} for r in runs]})
        print(i, n, insts[-1]["lstar"], flush=True)
    b = BATCH_SAMPLE
    out = {"workload": f"the first {b['take']} instances with n <= {b['max_n']} of the batched workload "
                       f"({b['count']} uniform instances, sizes log-uniform in [{b['lo']}, {b['hi']}] with "
                       f"size seed {b['size_seed']}, coordinate seed 1000 + index), m = n, cl = {b['cl']}, "
                       "alpha=1, beta=2, rho=0.02, p_best=0.01",
           "iterations": iters, "instances": insts, "source": "tests/golden/make_lstar.py (CPU oracle)"}
    with open(os.path.join(HERE, b["out"]), "w") as f:
        json.dump(out, f, indent=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batched-sample16"], default="uniform-n1000")
    ap.add_argument("--iters", type=int, default=None)
    ap.add_argument("--seeds", type=str, default=None, help="comma-separated MMAS seeds")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    if args.workload == "batched-sample16":
        return main_batch(args.iters or BATCH_SAMPLE["iters"], args.threads)
    w = WORKLOADS[args.workload]
    iters = args.iters or w["iters"]
    xy = instance(w)
    seeds = tuple(int(x) for x in args.seeds.split(",")) if args.seeds else w.get("seeds", (1, 2, 3))
    runs = []
    for seed in seeds:
        t0 = time.time()
        col = O.Colony(xy=xy, m=w["m"], cl=w["cl"], alpha=1.0, beta=2.0, rho=float(np.float32(0.02)),
                       p_best=float(np.float32(0.01)), seed=seed, ls=w["ls"])
        trace = []
        for it in range(iters):
            col.iterate(1, threads=args.threads)
            trace.append(int(col.best()[0]))
        runs.append({"seed": seed, "best": trace[-1], "trace_every_50": trace[49::50],
                     "seconds": round(time.time() - t0, 1)})
        print(seed, trace[-1], runs[-1]["seconds"], flush=True)
    out = {"workload": w["text"], "iterations": iters, "seeds": list(seeds),
           "lstar": min(r["best"] for r in runs), "runs": runs,
           "source": "tests/golden/make_lstar.py (CPU oracle)"}
    with open(os.path.join(HERE, w["out"]), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
