"""Small runs over every path of the library, for comparing the release build
with the -DGSB_DEBUG build (device-side bounds checks): the shapes are the
edge cases of the tiling (N = 1, 2, 17, 127, 129; R = 1, 3, plus a ragged
second replica block), each run reads its status word through best(), which
raises on a check that fired, and the results are written to an .npz for the
other build to compare bit for bit.

    python tests/_debug_cases.py OUT.npz     (GSB_LIBRARY=debug for the debug build)
"""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2508_17655_gb300 import gsb, inputs as I  # noqa: E402

SHAPES = [(1, 1), (2, 3), (17, 3), (127, 1), (129, 3), (129, 130)]


def _record(out, key, run):
    st = run.state()
    b = run.best()
    for k in ("x", "y", "p"):
        out[f"{key}/{k}"] = np.asarray(st[k])
    for k in ("E", "s", "step"):
        out[f"{key}/best_{k}"] = np.asarray(b[k])
    run.close()


def run_cases():
    out = {}
    kw = dict(M=30, dt=0.9, A=0.25, seed=11, eval_every=10)
    for N, R in SHAPES:
        Jpm = I.sk_pm1(N, 3) if N > 1 else np.zeros((1, 1), np.int8)
        Jg = I.sk_gauss(N, 3) if N > 1 else np.zeros((1, 1), np.float32)
        c = float(np.float32(1 / (2 * math.sqrt(N))))
        P = gsb.Problem.dense(Jpm)
        G = gsb.Problem.dense(Jg)
        for variant, prec in (("gdsb", "fp8"), ("dsb", "fp8"), ("gbsb", "fx32"), ("bsb", "fx32"),
                              ("gbsb", "fx16"), ("gbsb", "fp32"), ("gdsb", "fp32")):
            for spl in (0, 1) if prec == "fp8" else (0,):
                run = P.run(variant, R=R, c=c, precision=prec, steps_per_launch=spl, **kw)
                _record(out, f"dense/{N}/{R}/{variant}/{prec}/{spl}", run)
        for variant in ("gbsb", "gdsb"):
            run = G.run(variant, R=R, c=0.5, precision="bf16x3", **kw)
            _record(out, f"bf16/{N}/{R}/{variant}", run)
        if N >= 17:
            rp, col, val = I.er_graph(N, 4, "pm1", 7)
            C = gsb.Problem.csr(N, rp, col, val)
            for variant in ("gbsb", "gdsb"):
                for fused in (False, True):
                    run = C.run(variant, R=R, c=0.2, fused_csr=fused, **kw)
                    _record(out, f"csr/{N}/{R}/{variant}/{int(fused)}", run)
            C.close()
        P.close()
        G.close()
    # Lyapunov exponents and adjoint gradients, both coupling forms (the split
    # form's tangent step and K-split partial products included), at a ragged
    # shape: N = 129 (two spin tiles), 2 x 67 replicas (two replica tiles)
    import torch
    Jg = I.sk_gauss(129, 5)
    G = gsb.Problem.dense(Jg)
    x0 = I.uniform_state(67, 129, 4)
    xd = torch.from_numpy(np.ascontiguousarray(x0, dtype=np.float32)).cuda()
    for prec in ("fp32", "bf16x3"):
        for variant in ("gbsb", "gdsb"):
            out[f"lyap/{prec}/{variant}"] = np.asarray(
                G.lyapunov(variant, 400, 67, [0.1, 0.3], c=0.5, dt=0.9, seed=6, renorm_every=5,
                           nsteps=20, precision=prec))
            E = torch.empty(67, dtype=torch.float64, device="cuda")
            gx = torch.empty_like(xd)
            gA = torch.empty(67, dtype=torch.float64, device="cuda")
            gdt = torch.empty(67, dtype=torch.float64, device="cuda")
            G.relaxed_energy_grad(variant, 400, 9, xd.data_ptr(), 67, 0.2, 0.9, 0.5, E.data_ptr(),
                                  gx.data_ptr(), gA.data_ptr(), gdt.data_ptr(), ckpt_every=4,
                                  precision=prec)
            torch.cuda.synchronize()
            for k, t in (("E", E), ("gx", gx), ("gA", gA), ("gdt", gdt)):
                out[f"adj/{prec}/{variant}/{k}"] = t.cpu().numpy()
    G.close()
    # batched runs of uneven instances, both forms
    Ns, Rs = [17, 129, 64, 2], [3, 130, 1, 5]
    for form in ("fp32", "bf16x3"):
        probs, specs = [], []
        for k, (N, R) in enumerate(zip(Ns, Rs)):
            probs.append(gsb.Problem.dense(I.sk_gauss(N, 20 + k)))
            specs.append(dict(variant=("gbsb", "gdsb")[k % 2], M=20, R=R, c=0.5, dt=0.9,
                              A=0.2, seed=k, precision=form))
        runs, _ = gsb.batch_run(probs, specs)
        for k, run in enumerate(runs):
            _record(out, f"batch/{form}/{k}", run)
        for P in probs:
            P.close()
    return out


if __name__ == "__main__":
    res = run_cases()
    np.savez(sys.argv[1], **{k.replace("/", "|"): v for k, v in res.items()},
             debug_build=np.array(gsb.debug_build()))
    print(f"{len(res)} arrays, debug build {gsb.debug_build()}")
