"""Write the oracle's best-energy distributions on the N = 2000 workload.

Statistical parity (Sec. III measures the success probability P_S over many
runs from random initial conditions) at the dense precision workload: the
+-1 complete graph with N = 2000 (seed 0, the synthetic stand-in for K2000),
M = 2000 steps, dt = 1.25, c = 1/(2 sqrt N) (App. A), x(0) uniform in
[-0.1, 0.1), y(0) = 0 (App. A), energy at t_M only (Sec. III). For each
(variant, A) cell the FP64 oracle runs R = 1024 replicas and the final
energies are stored; the GPU test draws its own replicas (other seeds) and
compares P_S and the mean with two-sample bounds. This script calls only
oracle/ and the seeded generators.

    python tests/golden/make_stats_N2000.py [--threads T] [--quick]
"""
import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2508_17655_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "stats_N2000.json")

# (variant, A, seed): GdSB is the sgn-coupled form the FP8 kernels run, GbSB
# the paper's x-coupled form (FX32 kernels)
CELLS = [("gdsb", 0.1, 7001), ("gdsb", 0.25, 7002), ("gbsb", 0.2, 7003), ("gbsb", 0.25, 7004)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--quick", action="store_true")
    args = ap.parse_args()
    N, M, dt = 2000, 2000, 1.25
    R = 1024 if not args.quick else 8
    if args.quick:
        M = 50
    c = 1.0 / (2.0 * math.sqrt(N))
    J = I.sk_pm1(N, 0).astype(np.float64)
    out = {"N": N, "M": M, "dt": dt, "c": c, "R": R, "instance": "inputs.sk_pm1(2000, 0)",
           "x0": "oracle.init_uniform(R, N, seed), y0 = 0, p0 = 1", "cells": []}
    if os.path.exists(OUT) and not args.quick:
        with open(OUT) as f:
            old = json.load(f)
        if all(old.get(k) == out[k] for k in ("N", "M", "dt", "R")):
            out["cells"] = old["cells"]
    done = {(cl["variant"], cl["A"], cl["seed"]) for cl in out["cells"]}
    for variant, A, seed in CELLS:
        if (variant, A, seed) in done:
            continue
        x0 = O.init_uniform(R, N, seed)
        t = time.time()
        o = O.run(J, variant, x0, 0 * x0, c=c, dt=dt, M=M, A=A, eval_every=0,
                  nthreads=args.threads)
        E = o["best"]["E"]
        out["cells"].append({"variant": variant, "A": A, "seed": seed,
                             "energies": [int(round(e)) for e in E.tolist()],
                             "seconds": round(time.time() - t, 1)})
        print(variant, A, "mean", float(E.mean()), "min", float(E.min()),
              round(time.time() - t, 1), "s", flush=True)
        if not args.quick:
            with open(OUT + ".tmp", "w") as f:
                json.dump(out, f, separators=(",", ":"))
            os.replace(OUT + ".tmp", OUT)
    print("wrote", OUT if not args.quick else "(quick: nothing)")


if __name__ == "__main__":
    main()
