"""Write the target energies used for success probability and TTS99.

The synthetic instances have no published best-known value (the paper's K2000
best cut, Sec. III, belongs to a different instance). The target of each
instance is the lowest energy found by long FP64 oracle runs (GbSB, Eq. 7, and
dSB, Sec. VI, at several control strengths and step counts), recorded with how
often it was hit. This script calls only oracle/ and the seeded generators.

    python tests/golden/make_targets.py [--quick]
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

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "targets.json")


def long_runs(J, N, variants, R, M, dt, c, seed0, threads):
    found = []
    for k, (variant, A) in enumerate(variants):
        x0 = O.init_uniform(R, N, seed0 + k)
        t = time.time()
        o = O.run(J, variant, x0, 0 * x0, c=c, dt=dt, M=M, A=A, eval_every=0, nthreads=threads)
        found.append({"variant": variant, "A": A, "M": M, "R": R, "seed": seed0 + k,
                      "energies": sorted(o["best"]["E"].tolist())[:8],
                      "min": float(o["best"]["E"].min()), "seconds": round(time.time() - t, 1)})
        print(found[-1]["variant"], A, M, found[-1]["min"], found[-1]["seconds"], flush=True)
    return found


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    targets = {}
    # config 1: N = 100 SK +-1, seed 0, dt = 0.5, c = 0.05 (App. A estimate 1/(2 sqrt N))
    N = 100
    J = I.sk_pm1(N, 0).astype(np.float64)
    runs = long_runs(J, N, [("gbsb", 0.2), ("gbsb", 0.3), ("dsb", 0.0), ("gdsb", 0.2)],
                     256 if not args.quick else 32, 20000 if not args.quick else 2000, 0.5, 0.05,
                     100, args.threads)
    e = min(r["min"] for r in runs)
    targets["sk_pm1_N100_seed0"] = {"N": N, "E_target": e, "W_tot": O.total_weight(J),
                                    "runs": runs, "how": "min over the long oracle runs listed"}
    # config 2: N = 2000 complete graph +-1, seed 0, dt = 1.25, c = 1/(2 sqrt N)
    N = 2000
    J = I.sk_pm1(N, 0).astype(np.float64)
    c = 1.0 / (2.0 * math.sqrt(N))
    R = 32 if not args.quick else 4
    M = 10000 if not args.quick else 500
    runs = long_runs(J, N, [("gbsb", 0.2), ("gbsb", 0.25), ("gdsb", 0.2), ("dsb", 0.0)], R, M,
                     1.25, c, 200, args.threads)
    e = min(r["min"] for r in runs)
    targets["sk_pm1_N2000_seed0"] = {"N": N, "E_target": e, "W_tot": O.total_weight(J),
                                     "cut_target": (O.total_weight(J) - e) / 2, "runs": runs,
                                     "how": "min over the long oracle runs listed"}
    with open(OUT, "w") as f:
        json.dump(targets, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
