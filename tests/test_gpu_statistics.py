"""Statistical parity over the whole run, where chaos has long decorrelated
individual trajectories: success probability P_S and mean best energy of
>= 1000 replicas on the GPU against the FP64 oracle, each within its 99 %
confidence bound (two-proportion z bound for P_S, Welch bound for the mean).

Workload: the small dense configuration (N = 100 SK, i.i.d. +-1, seed 0;
x, y uniform in [-0.1, 0.1); M = 1000; dt = 0.5; c = 0.05), target energy from
long oracle runs (tests/golden/targets.json)."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2508_17655_gb300 import gsb, inputs as I

pytestmark = pytest.mark.gpu

Z99 = 2.5758293035489  # two-sided 99 % normal quantile


def _target(key):
    path = os.path.join(os.path.dirname(__file__), "golden", "targets.json")
    with open(path) as f:
        return json.load(f)[key]["E_target"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build()


def _compare(e_gpu, e_ref, target):
    n1, n2 = len(e_gpu), len(e_ref)
    p1 = float(np.mean(e_gpu <= target))
    p2 = float(np.mean(e_ref <= target))
    pbar = (p1 * n1 + p2 * n2) / (n1 + n2)
    bound_p = Z99 * math.sqrt(max(pbar * (1 - pbar), 0.0) * (1 / n1 + 1 / n2))
    assert abs(p1 - p2) <= bound_p + 1e-12, f"P_S gpu {p1:.4f} vs oracle {p2:.4f} (bound {bound_p:.4f})"
    m1, m2 = float(np.mean(e_gpu)), float(np.mean(e_ref))
    bound_m = Z99 * math.sqrt(np.var(e_gpu, ddof=1) / n1 + np.var(e_ref, ddof=1) / n2)
    assert abs(m1 - m2) <= bound_m + 1e-9, f"mean E gpu {m1:.3f} vs oracle {m2:.3f} (bound {bound_m:.3f})"
    return p1, p2, m1, m2


@pytest.mark.parametrize("variant,precision,A", [("gbsb", "auto", 0.2), ("gbsb", "fp32", 0.2),
                                                 ("gdsb", "auto", 0.2), ("dsb", "auto", 0.0),
                                                 ("bsb", "auto", 0.0)])
def test_success_probability_and_mean_energy_config1(variant, precision, A):
    N, R, M, dt = 100, 1024, 1000, 0.5
    c = float(np.float32(0.05))
    J = I.sk_pm1(N, 0)
    target = _target("sk_pm1_N100_seed0")
    run = gsb.Problem.dense(J).run(variant, M=M, R=R, c=c, dt=dt, A=A, seed=77, y0_uniform=True,
                                   precision=precision)
    e_gpu = run.best()["E"]
    x0 = O.init_uniform(R, N, 77)
    y0 = O.init_uniform(R, N, 77, stream=1)
    ref = O.run(J.astype(np.float64), variant, x0, y0, c=c, dt=dt, M=M, A=A)
    e_ref = ref["best"]["E"]
    assert np.all(e_gpu >= target) and np.all(e_ref >= target)  # nobody beats the target
    _compare(e_gpu, e_ref, target)


@pytest.mark.parametrize("variant", ["gbsb", "gdsb"])
def test_mean_best_energy_sparse(variant):
    """Sparse ER instance (N = 1000, mean degree 20, +-1 weights), 1024
    replicas, 800 steps, c = 1/lambda_max, dt from Eq. 13: mean best energy
    within the 99 % Welch bound; P_S against the best energy either side saw
    is not used (no independent target for this instance)."""
    N, R, M = 1000, 1024, 800
    rp, col, val = I.er_graph(N, 20, "pm1", 11)
    C = O.Coupling(N, rowptr=rp, col=col, val=val)
    lmax, lmin = O.lambda_extremes(C)
    c = float(np.float32(1 / lmax))
    dt = float(np.float32(O.dt_from_lambda(lmax, lmin)))
    run = gsb.Problem.csr(N, rp, col, val).run(variant, M=M, R=R, c=c, dt=dt, A=0.2, seed=5)
    e_gpu = run.best()["E"]
    x0 = O.init_uniform(R, N, 5)
    e_ref = O.run(C, variant, x0, 0 * x0, c=c, dt=dt, M=M, A=0.2)["best"]["E"]
    m1, m2 = float(np.mean(e_gpu)), float(np.mean(e_ref))
    bound = Z99 * math.sqrt(np.var(e_gpu, ddof=1) / R + np.var(e_ref, ddof=1) / R)
    assert abs(m1 - m2) <= bound, f"mean E gpu {m1:.3f} vs oracle {m2:.3f} (bound {bound:.3f})"


def _stats_golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "stats_N2000.json")
    with open(path) as f:
        return json.load(f)


def _cells():
    """(variant, A, precision) of every cell: "auto" and "fp32" for each variant,
    and FX16 (the x coupling's 16-bit form) for the x-coupled variants."""
    out = []
    for c in _stats_golden()["cells"]:
        for precision in ("auto", "fp32", "fx16"):
            if precision != "fx16" or c["variant"] in ("gbsb", "bsb"):
                out.append((c["variant"], c["A"], precision))
    return out


@pytest.mark.parametrize("variant,A,precision", _cells())
def test_headline_shape_statistics_match_oracle(variant, A, precision):
    """The dense precision workload itself: N = 2000 +-1 complete graph (seed
    0), M = 2000, dt = 1.25, c = 1/(2 sqrt N), R = 1024 replicas from x(0)
    uniform in [-0.1, 0.1), y(0) = 0 (App. A), energy at t_M (Sec. III). The
    FP64 oracle's 1024 final energies per (variant, A) come from
    tests/golden/make_stats_N2000.py; the GPU draws its own 1024 replicas
    (another seed) on the path the bench times ("auto": the persistent FP8
    kernel for GdSB, FX32 digit planes for GbSB), on the plain FP32 form, and
    for GbSB on the paper's 16-bit fixed-point JX (FX16), whose x grid of
    2^-15 leaves the statistics of the FP64 run unchanged within the bounds.
    Within the 99 % bounds: P_S at the oracle target energy (two-proportion),
    P(E <= the oracle's median energy), and the mean best energy (Welch)."""
    g = _stats_golden()
    cell = next(c for c in g["cells"] if c["variant"] == variant and c["A"] == A)
    e_ref = np.asarray(cell["energies"], dtype=np.float64)
    N, R, M, dt = g["N"], g["R"], g["M"], g["dt"]
    c = float(np.float32(g["c"]))
    run = gsb.Problem.dense(I.sk_pm1(N, 0)).run(variant, M=M, R=R, c=c, dt=dt, A=A,
                                                 seed=88000 + int(1000 * A), precision=precision)
    if precision == "auto":
        assert run.kernel().startswith("k_tc_persist" if variant == "gdsb" else "k_fx32")
    if precision == "fx16":
        assert run.kernel() == "k_fx16_persist"
    e_gpu = run.best()["E"]
    target = _target("sk_pm1_N2000_seed0")
    _compare(e_gpu, e_ref, target)
    _compare(e_gpu, e_ref, float(np.median(e_ref)))
