"""Write the target energies used for success probability and TTS99.

The synthetic instances have no published best-known value (the paper's K2000
best cut, Sec. III, belongs to a different instance). The target of each
instance is the lowest energy found by long FP64 oracle runs (GbSB, Eq. 7, and
dSB, Sec. VI, at several control strengths and step counts), recorded with how
often it was hit. This script calls only oracle/ and the seeded generators.

For the N = 2000 complete graph the long runs use the paper's own K2000
setting (Fig. 1(d): M = 21,500 at dt = 1.25, A = 0.2 and 0.25) and GdSB at
M = 20,000; batches of replicas are added until the lowest energy has been
reached at least three times (or the time budget is spent), and every batch
is recorded.

    python tests/golden/make_targets.py [--quick] [--only N100|N2000] [--budget-s S]
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


def one_batch(J, N, variant, A, R, M, dt, c, seed, threads):
    x0 = O.init_uniform(R, N, seed)
    t = time.time()
    o = O.run(J, variant, x0, 0 * x0, c=c, dt=dt, M=M, A=A, eval_every=0, nthreads=threads)
    E = o["best"]["E"]
    rec = {"variant": variant, "A": A, "M": M, "R": R, "seed": seed,
           "energies": sorted(E.tolist()), "min": float(E.min()),
           "seconds": round(time.time() - t, 1)}
    print(variant, A, M, R, seed, rec["min"], rec["seconds"], flush=True)
    return rec


def long_runs(J, N, variants, R, M, dt, c, seed0, threads):
    return [one_batch(J, N, v, A, R, M, dt, c, seed0 + k, threads)
            for k, (v, A) in enumerate(variants)]


def load():
    if os.path.exists(OUT):
        with open(OUT) as f:
            return json.load(f)
    return {}


def save(targets):
    with open(OUT + ".tmp", "w") as f:
        json.dump(targets, f, indent=1)
    os.replace(OUT + ".tmp", OUT)


def target_n100(args, targets):
    # config 1: N = 100 SK +-1, seed 0, dt = 0.5, c = 0.05 (App. A estimate 1/(2 sqrt N))
    N = 100
    J = I.sk_pm1(N, 0).astype(np.float64)
    runs = long_runs(J, N, [("gbsb", 0.2), ("gbsb", 0.3), ("dsb", 0.0), ("gdsb", 0.2)],
                     256 if not args.quick else 32, 20000 if not args.quick else 2000, 0.5, 0.05,
                     100, args.threads)
    for r in runs:
        r["energies"] = r["energies"][:8]
    e = min(r["min"] for r in runs)
    targets["sk_pm1_N100_seed0"] = {"N": N, "E_target": e, "W_tot": O.total_weight(J),
                                    "runs": runs, "how": "min over the long oracle runs listed"}


def target_n2000(args, targets):
    # config 2: N = 2000 complete graph +-1, seed 0, dt = 1.25, c = 1/(2 sqrt N) (App. A)
    N = 2000
    J = I.sk_pm1(N, 0).astype(np.float64)
    c = 1.0 / (2.0 * math.sqrt(N))
    R = 32 if not args.quick else 4
    settings = [("gbsb", 0.2, 21500), ("gbsb", 0.25, 21500), ("gdsb", 0.2, 20000)]
    if args.quick:
        settings = [(v, A, 300) for v, A, _ in settings]
    key = "sk_pm1_N2000_seed0"
    old = targets.get(key, {})
    runs = [r for r in old.get("runs", []) if r["M"] >= 20000] if not args.quick else []
    seed = max([r["seed"] for r in runs] + [299]) + 1
    t0 = time.time()

    def summary():
        allE = np.concatenate([np.asarray(r["energies"]) for r in runs])
        e = float(allE.min())
        return e, int(np.sum(allE <= e + 1e-9)), int(allE.size)

    # the paper's GbSB setting is run once per (A, M); the batches added until
    # the lowest energy has three hits are GdSB, which reaches it far more often
    # on this instance (Sec. VII names the control with the sgn coupling as a
    # direction)
    done = {(r["variant"], r["A"], r["M"]) for r in runs}
    while True:
        todo = [(v, A, M) for v, A, M in settings if v != "gbsb" or (v, A, M) not in done]
        for v, A, M in todo:
            done.add((v, A, M))
            runs.append(one_batch(J, N, v, A, R, M, 1.25, c, seed, args.threads))
            seed += 1
            e, hits, n = summary()
            targets[key] = {
                "N": N, "E_target": e, "W_tot": O.total_weight(J),
                "cut_target": (O.total_weight(J) - e) / 2, "hits": hits, "replicas": n,
                "runs": runs,
                "how": ("lowest energy of the long oracle runs listed (M >= 20,000; "
                        "the paper's K2000 setting M = 21,500, dt = 1.25, Fig. 1(d)), "
                        "with the number of replicas that reached it"),
            }
            save(targets)
        e, hits, n = summary()
        print("target", e, "hits", hits, "of", n, flush=True)
        if hits >= 3 or time.time() - t0 > args.budget_s or args.quick:
            break


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--only", choices=["N100", "N2000"], default=None)
    ap.add_argument("--budget-s", type=float, default=4 * 3600.0)
    args = ap.parse_args()
    targets = load()
    if args.only in (None, "N100"):
        target_n100(args, targets)
        save(targets)
    if args.only in (None, "N2000"):
        target_n2000(args, targets)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
