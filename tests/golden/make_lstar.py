"""Write the oracle's long-run best tour length L* of a benchmark workload.

L* is the shortest tour the CPU oracle (MMAS, Alg. 1) finds over MMAS seeds
1..3, each run for the workload's full iteration budget, with alpha = 1,
beta = 2, rho = 0.02, p_best = 0.01.  It anchors the time-to-within-2%
measurement.  Calls only the oracle.  Workloads:

  uniform-n1000   synthetic uniform n = 1000 (coordinate seed 1001), m = 1000,
                  cl = 32, 1000 iterations -> lstar_uniform_n1000.json
  clustered-n3800 synthetic clustered n = 3800 (seed 1003), m = 1000, cl = 16,
                  2-opt of each iteration's best (Sec. 5.7), 500 iterations
                  -> lstar_clustered_n3800.json

    python tests/golden/make_lstar.py [--workload uniform-n1000] [--iters N] [--threads N]
"""
import argparse
import json
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
    "clustered-n3800": dict(kind="clustered", n=3800, iseed=1003, m=1000, cl=16, ls=1, iters=500,
                            out="lstar_clustered_n3800.json",
                            text="clustered n=3800 (seed 1003), m=1000, cl=16, 2-opt of the iteration "
                                 "best, alpha=1, beta=2, rho=0.02, p_best=0.01"),
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="uniform-n1000")
    ap.add_argument("--iters", type=int, default=None)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    iters = args.iters or w["iters"]
    xy = I.uniform(w["n"], w["iseed"]) if w["kind"] == "uniform" else I.clustered(w["n"], w["iseed"])
    runs = []
    for seed in (1, 2, 3):
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
    out = {"workload": w["text"], "iterations": iters,
           "lstar": min(r["best"] for r in runs), "runs": runs,
           "source": "tests/golden/make_lstar.py (CPU oracle)"}
    with open(os.path.join(HERE, w["out"]), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
