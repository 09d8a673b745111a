"""Write the oracle's long-run best tour length L* for the n = 1000 workload.

L* is the shortest tour the CPU oracle (MMAS, Alg. 1) finds on the synthetic
uniform n = 1000 instance (coordinate seed 1001) with m = 1000 ants, cl = 32,
alpha = 1, beta = 2, rho = 0.02, p_best = 0.01, over MMAS seeds 1..3, each run
for the workload's full budget of 1000 iterations.  It anchors the
time-to-within-2% measurement.  Calls only the oracle.

    python tests/golden/make_lstar.py [--iters 1000] [--threads N]
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=1000)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    xy = I.uniform(1000, 1001)
    runs = []
    for seed in (1, 2, 3):
        t0 = time.time()
        col = O.Colony(xy=xy, m=1000, cl=32, alpha=1.0, beta=2.0, rho=float(np.float32(0.02)),
                       p_best=float(np.float32(0.01)), seed=seed)
        trace = []
        for it in range(args.iters):
            col.iterate(1, threads=args.threads)
            trace.append(int(col.best()[0]))
        runs.append({"seed": seed, "best": trace[-1], "trace_every_50": trace[49::50],
                     "seconds": round(time.time() - t0, 1)})
        print(seed, trace[-1], runs[-1]["seconds"], flush=True)
    out = {"workload": "uniform n=1000 (coordinate seed 1001), m=1000, cl=32, alpha=1, beta=2, "
                       "rho=0.02, p_best=0.01", "iterations": args.iters,
           "lstar": min(r["best"] for r in runs), "runs": runs,
           "source": "tests/golden/make_lstar.py (CPU oracle)"}
    with open(os.path.join(HERE, "lstar_uniform_n1000.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
