"""The split-bf16 tensor-core path for real-valued couplings (GSB_PREC_BF16X3,
the default for non-integer dense J): J = J_hi + J_lo and x = x_hi + x_lo in
bf16, three products accumulated in FP32 (two for the sgn coupling), one
persistent launch per stretch of steps.

Against the FP64 oracle: one re-synchronised step within 1e-4 of each
update's operand magnitudes (the split's residue is at most 3 x 2^-16 =
4.6e-5 of sum_j |J_ij x_j|, plus FP32 accumulation); the first 50 steps'
error reported and bounded; energies exactly those of the reported spins. The
schedule (steps per launch, grid) does not change a bit of the result."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2508_17655_gb300 import gsb, inputs as I
from tests._parity import assert_one_step_close, coupling_scale_drift, note_widened

pytestmark = pytest.mark.gpu

EPS_BF16 = 1e-4
VARIANTS = ["bsb", "gbsb", "dsb", "gdsb"]


def f32(v):
    return float(np.float32(v))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build()


def test_real_J_defaults_to_the_split_bf16_path():
    P = gsb.Problem.dense(I.sk_gauss(200, 1))
    for v in VARIANTS:
        assert P.run(v, M=10, R=8, c=0.5, dt=1.0, defer=True).kernel() == "k_bf16_multi"
    # integer couplings keep their exact forms by default
    Q = gsb.Problem.dense(I.sk_pm1(200, 1))
    assert Q.run("gbsb", M=10, R=8, c=0.05, dt=1.0, defer=True).kernel().startswith("k_fx32")


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("N,R", [(300, 200), (129, 1), (1000, 129), (2000, 1024)])
def test_bf16_one_step_resync_within_split_bar(variant, N, R):
    """SK N(0, 1/N) couplings, c = 1/2 (App. A), dt = 1.25: at steps 0, 37 and
    the last of M = 400 the GPU state is handed to the oracle and both advance
    one step; every element within EPS_BF16 of its update's operand
    magnitudes. N = 2000, R = 1024 is the chaos configuration's size class."""
    M = 400
    J = I.sk_gauss(N, 7)
    Jo = J.astype(np.float64)
    P = gsb.Problem.dense(J)
    run = P.run(variant, M=M, R=R, c=0.5, dt=1.25, A=0.25, seed=3, precision="bf16x3",
                defer=True)
    done = 0
    for m in (0, 37, M - 1):
        if m > done:
            run.steps(m - done)
        s0 = run.state()
        run.steps(1)
        done = m + 1
        s1 = run.state()
        ref = O.run(Jo, variant, s0["x"].astype(np.float64), s0["y"].astype(np.float64),
                    c=0.5, dt=1.25, M=M, A=0.25, p=s0["p"].astype(np.float64), m0=m, nsteps=1)
        assert_one_step_close(s0, s1, ref, Jo, variant, 0.5, 1.25, ref["wall_margin"],
                              eps=EPS_BF16, what=f"bf16 {variant} N={N} m={m}")


@pytest.mark.parametrize("variant", ["gbsb", "bsb"])
def test_bf16_first_50_steps_error(variant):
    """N = 1000 SK, R = 256, M = 1000: norm-wise error of x against the FP64
    oracle after 50 steps, for 16 sampled replicas, recorded, and within 3x the
    drift that a systematic coupling error of the split's residue size (2^-16
    relative) causes in the oracle by itself. The instability of the top modes
    (c lambda_max >= 1) amplifies coupling errors coherently here: 1e-5 of the
    coupling becomes 1e-3 to 7e-3 of x in 50 steps; the FP32 CUDA-core form,
    with residues near 2^-24, stays near 1e-4. (For the sgn couplings the
    comparison over 50 steps is dominated by sign decisions taken differently
    near x = 0; the one-step test above covers them element by element.)"""
    N, R, M = 1000, 256, 1000
    J = I.sk_gauss(N, 11)
    Jo = J.astype(np.float64)
    run = gsb.Problem.dense(J).run(variant, M=M, R=R, c=0.5, dt=1.25, A=0.2, seed=5, defer=True)
    run.steps(50)
    st = run.state()
    pick = np.linspace(0, R - 1, 16).astype(int)
    x0 = O.init_uniform(R, N, 5)[pick]
    ref, drift = coupling_scale_drift(
        lambda x, scale, n: O.run(Jo, variant, x, 0 * x, c=0.5 * scale, dt=1.25, M=M, A=0.2,
                                  nsteps=n), x0, 50)
    ok = ref["margin"] >= 2e-6
    err = np.linalg.norm(st["x"][pick] - ref["x"], axis=1) / np.linalg.norm(ref["x"], axis=1)
    note_widened(f"bf16 50 steps {variant}: worst {float(err[ok].max()):.2e}, residue drift "
                 f"{float(drift.max()):.2e}", int((~ok).sum()), len(ok),
                 "excused: near-tie decision")
    assert ok.sum() >= 8
    bad = ok & (err > np.maximum(1e-5, 3.0 * drift))
    assert not bad.any(), (err[bad], drift[bad])


@pytest.mark.parametrize("variant", ["gbsb", "dsb"])
def test_bf16_schedule_does_not_change_bits(variant):
    """One launch for the run, a launch every 7 steps, and energies every 25
    steps (launches cut at each): identical state and best records."""
    N, R, M = 700, 300, 120
    P = gsb.Problem.dense(I.sk_gauss(N, 13))
    outs = []
    for spl, ev in ((0, 0), (7, 0), (0, 25)):
        run = P.run(variant, M=M, R=R, c=0.5, dt=1.0, A=0.3, seed=2, steps_per_launch=spl,
                    eval_every=ev)
        outs.append((run.state(), run.best()))
    for st, b in outs[1:]:
        for k in ("x", "y", "p"):
            assert np.array_equal(st[k], outs[0][0][k]), k
        assert np.array_equal(b["E"][b["step"] == M], outs[0][1]["E"][b["step"] == M])


def test_bf16_energies_are_those_of_the_reported_spins():
    N, R, M = 500, 200, 300
    J = I.sk_gauss(N, 17)
    run = gsb.Problem.dense(J).run("gbsb", M=M, R=R, c=0.5, dt=1.25, A=0.2, seed=1,
                                   eval_every=50)
    b = run.best()
    np.testing.assert_allclose(b["E"], O.energy(J.astype(np.float64), b["s"]), rtol=1e-6,
                               atol=1e-6)
    assert np.all((b["step"] % 50 == 0) & (b["step"] > 0))


@pytest.mark.parametrize("kind", ["fp8", "fx32", "bf16x3"])
def test_resume_at_an_odd_step_is_bit_exact(kind):
    """A run saved after an odd number of steps (51) and restored into a fresh
    run continues exactly as the uninterrupted run: the restored operand goes
    to the buffer of the step's parity, which the persistent kernels read."""
    M, R, k = 120, 200, 51
    if kind == "bf16x3":
        P, variant, c = gsb.Problem.dense(I.sk_gauss(300, 4)), "gdsb", 0.5
    else:
        P, variant, c = gsb.Problem.dense(I.sk_pm1(300, 4)), ("gdsb" if kind == "fp8" else "gbsb"), 0.03
    kw = dict(M=M, R=R, c=c, dt=1.0, A=0.3, seed=12, precision=kind)
    whole = P.run(variant, **kw)
    want = whole.state()
    part = P.run(variant, defer=True, **kw)
    part.steps(k)
    saved = part.state()
    fresh = P.run(variant, defer=True, **kw)
    fresh.set_state(saved)
    fresh.steps(M - k)
    got = fresh.state()
    for key in ("x", "y", "p"):
        assert np.array_equal(got[key], want[key]), key
