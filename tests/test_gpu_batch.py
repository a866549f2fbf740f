"""Batched runs of uneven instances (gsb_batch_run): each instance follows
the trajectory it follows alone, whatever tile the autotuner picks, and its
error against the FP64 oracle stays within the single-run bars."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2508_17655_gb300 import gsb, inputs as I
from tests._parity import assert_one_step_close

pytestmark = pytest.mark.gpu


def f32(v):
    return float(np.float32(v))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build()


def _instances():
    Ns = [70, 129, 200, 257, 300, 64, 100, 511, 128, 90]
    Rs = [33, 64, 100, 129, 40, 200, 17, 50, 128, 77]
    variants = ["gbsb", "gdsb", "bsb", "dsb", "gbsb", "gdsb", "gbsb", "dsb", "bsb", "gbsb"]
    Ms = [120, 120, 80, 120, 100, 120, 120, 60, 120, 95]
    probs, specs = [], []
    for k, (N, R, v, M) in enumerate(zip(Ns, Rs, variants, Ms)):
        J = I.sk_gauss(N, 100 + k) if k % 2 == 0 else I.sk_pm1(N, 100 + k)
        probs.append(gsb.Problem.dense(J))
        c = f32(0.5 if k % 2 == 0 else 1 / (2 * math.sqrt(N)))
        specs.append(dict(variant=v, M=M, R=R, c=c, dt=f32(1.0), A=0.1 + 0.02 * k, seed=7 + k))
    return probs, specs


@pytest.mark.parametrize("force", [0, 128, 64])
def test_batched_instances_match_their_single_runs_bit_exact(force):
    probs, specs = _instances()
    runs, info = gsb.batch_run(probs, specs, force_tile=force)
    if force:
        assert info["tile"] == force
    for P, sp, run in zip(probs, specs, runs):
        alone = P.run(precision="fp32", **sp)
        a, b = run.state(), alone.state()
        for k in ("x", "y", "p"):
            assert np.array_equal(a[k], b[k]), (sp, k)
        ba, bb = run.best(), alone.best()
        assert np.array_equal(ba["E"], bb["E"]) and np.array_equal(ba["s"], bb["s"])
        assert np.all(ba["step"] == sp["M"])


def test_batched_config4_shape_one_step_parity():
    """Config-4 shape: SK instances with N ~ U{64..1024}, Gaussian couplings
    N(0, 1/N), R ~ U{32..256}, c = 1/2, dt = 1.25, M = 1000. For every instance,
    the batched kernel's step m -> m+1 (m = 0 and 37) against the FP64 oracle
    started from the batched kernel's FP32 state at m: every element within
    1e-5 of its update's operand magnitudes (the single-run bar)."""
    Ns, Rs = I.batch_sizes(12, seed=4)
    probs, specs, Js = [], [], []
    for k, (N, R) in enumerate(zip(Ns.tolist(), Rs.tolist())):
        J = I.sk_gauss(N, 1000 + k)
        Js.append(J.astype(np.float64))
        probs.append(gsb.Problem.dense(J))
        specs.append(dict(variant="gbsb", M=1000, R=R, c=0.5, dt=1.25, A=0.2, seed=k))
    for m in (0, 37):
        s0 = [r.state() for r in gsb.batch_run(probs, specs, max_steps=m)[0]] if m else None
        s1 = [r.state() for r in gsb.batch_run(probs, specs, max_steps=m + 1)[0]]
        for k in range(len(probs)):
            N, R = int(Ns[k]), int(Rs[k])
            if m == 0:
                x0 = O.init_uniform(R, N, k)
                st0 = {"x": x0, "y": 0 * x0, "p": np.ones_like(x0)}
            else:
                st0 = s0[k]
            ref = O.run(Js[k], "gbsb", np.asarray(st0["x"], np.float64),
                        np.asarray(st0["y"], np.float64), c=0.5, dt=1.25, M=1000, A=0.2,
                        p=np.asarray(st0["p"], np.float64), m0=m, nsteps=1)
            assert_one_step_close(st0, s1[k], ref, Js[k], "gbsb", 0.5, 1.25, ref["margin"],
                                  what=f"instance {k} (N={N}, R={R}) m={m}")


def test_batched_config4_shape_50_step_error_and_energies():
    """The same instances over the first 50 steps: per-instance error against
    the FP64 oracle (sampled replicas), which FP32 sequential coupling sums and
    the instability of the top modes (c lambda_max >= 1 for these N) grow to
    ~1e-4 on some instances -- bounded here by 1e-3 -- and after finishing each
    run alone, best energies equal to the oracle energies of the best spins."""
    Ns, Rs = I.batch_sizes(12, seed=4)
    probs, specs, Js = [], [], []
    for k, (N, R) in enumerate(zip(Ns.tolist(), Rs.tolist())):
        J = I.sk_gauss(N, 1000 + k)
        Js.append(J.astype(np.float64))
        probs.append(gsb.Problem.dense(J))
        specs.append(dict(variant="gbsb", M=1000, R=R, c=0.5, dt=1.25, A=0.2, seed=k))
    runs, info = gsb.batch_run(probs, specs, max_steps=50)
    worst = 0.0
    for k, run in enumerate(runs):
        N, R = int(Ns[k]), int(Rs[k])
        st = run.state()
        assert st["steps"] == 50
        pick = np.linspace(0, R - 1, 4).astype(int)
        x0 = O.init_uniform(R, N, k)[pick]
        ref = O.run(Js[k], "gbsb", x0, 0 * x0, c=0.5, dt=1.25, M=1000, A=0.2, nsteps=50)
        ok = ref["margin"] >= 2e-6
        err = np.linalg.norm(st["x"][pick] - ref["x"], axis=1) / np.linalg.norm(ref["x"], axis=1)
        worst = max(worst, float(err[ok].max()) if ok.any() else 0.0)
        run.steps(950)  # finish the run alone; energies at t_M
        b = run.best()
        np.testing.assert_allclose(b["E"], O.energy(Js[k], b["s"]), rtol=1e-6, atol=1e-6)
    print(f"worst per-instance 50-step error vs FP64: {worst:.2e}")
    assert worst <= 1e-3
