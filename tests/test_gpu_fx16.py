"""FX16 (GSB_PREC_FX16): the x coupling on the 16-bit fixed-point grid of the
paper's JX module (Sec. VI, Fig. 2 caption), q = rint(x 2^15) as four e4m3
digit planes in two exact FP32 accumulators, one persistent launch with x, y
in TMEM and p in shared memory.

The oracle reads the same passage (oracle.run(..., jx16=True): x rounded to
the 2^-15 grid in the coupling only, FP64 everywhere else), so the FP32
trajectory bars of the exact paths apply: one re-synchronised step within
1e-5 of each update's operand magnitudes (element by element, on the timed
shape N = 2000, R = 1024), the first 50 steps within 1e-5 or 3x the FP32
storage drift."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2508_17655_gb300 import gsb, inputs as I
from tests._parity import (RTOL_TRAJ, assert_one_step_close, assert_within_fp32_drift,
                           fp32_storage_drift)

pytestmark = pytest.mark.gpu


def f32(v):
    return float(np.float32(v))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build()


@pytest.mark.parametrize("variant", ["gbsb", "bsb"])
@pytest.mark.parametrize("N,R", [(2000, 1024), (300, 200), (129, 1), (130, 129)])
def test_fx16_one_step_resync_every_element(variant, N, R):
    M, A = 2000, 0.25
    J = I.sk_pm1(N, 0 if N == 2000 else 21)
    Jo = J.astype(np.float64)
    c = f32(1 / (2 * math.sqrt(N)))
    run = gsb.Problem.dense(J).run(variant, M=M, R=R, c=c, dt=1.25, A=A, seed=23,
                                   precision="fx16", defer=True)
    assert run.kernel() == "k_fx16_persist"
    done = 0
    for m in (0, 50, 1000, 1999):
        if m > done:
            run.steps(m - done)
        s0 = run.state()
        run.steps(1)
        done = m + 1
        s1 = run.state()
        ref = O.run(Jo, variant, s0["x"].astype(np.float64), s0["y"].astype(np.float64),
                    c=c, dt=1.25, M=M, A=A, p=s0["p"].astype(np.float64), m0=m, nsteps=1,
                    jx16=True)
        assert_one_step_close(s0, s1, ref, Jo, variant, c, 1.25, ref["wall_margin"],
                              what=f"fx16 {variant} N={N} m={m}")


@pytest.mark.parametrize("variant", ["gbsb", "bsb"])
def test_fx16_first_50_steps_k2000_shape(variant):
    """N = 2000, R = 1024, M = 2000, dt = 1.25: 16 sampled replicas after 50
    steps within 1e-5 (norm-wise) of the oracle's 16-bit-JX trajectory, or 3x
    the drift FP32 storage of the state causes by itself."""
    N, R, M, A = 2000, 1024, 2000, 0.25
    J = I.sk_pm1(N, 0)
    Jo = J.astype(np.float64)
    c = f32(1 / (2 * math.sqrt(N)))
    run = gsb.Problem.dense(J).run(variant, M=M, R=R, c=c, dt=1.25, A=A, seed=9,
                                   precision="fx16", defer=True)
    run.steps(50)
    st = run.state()
    pick = np.linspace(0, R - 1, 16).astype(int)
    x0 = O.init_uniform(R, N, 9)[pick]
    ref, drift = fp32_storage_drift(
        lambda x, y, p, m0, n: O.run(Jo, variant, x, y, p=p, c=c, dt=1.25, M=M, A=A, m0=m0,
                                     nsteps=n, jx16=True), x0, 50)
    assert_within_fp32_drift(st["x"][pick], ref, drift, RTOL_TRAJ)


def test_fx16_schedule_does_not_change_bits():
    """One launch, a launch every 7 steps, and energies every 25 steps: the
    digit sums are exact, so the results are identical."""
    N, R, M = 500, 256, 120
    P = gsb.Problem.dense(I.sk_pm1(N, 13))
    outs = []
    for spl, ev in ((0, 0), (7, 0), (0, 25)):
        run = P.run("gbsb", M=M, R=R, c=0.02, dt=1.0, A=0.3, seed=2, precision="fx16",
                    steps_per_launch=spl, eval_every=ev)
        outs.append(run.state())
    for st in outs[1:]:
        for k in ("x", "y", "p"):
            assert np.array_equal(st[k], outs[0][k]), k


def test_fx16_energies_and_rejections():
    N, R, M = 300, 130, 200
    J = I.sk_pm1(N, 17)
    P = gsb.Problem.dense(J)
    run = P.run("gbsb", M=M, R=R, c=0.03, dt=1.0, A=0.2, seed=1, precision="fx16", eval_every=40)
    b = run.best()
    np.testing.assert_array_equal(b["E"], O.energy(J.astype(np.float64), b["s"]))
    assert np.all((b["step"] % 40 == 0) & (b["step"] > 0))
    for variant in ("dsb", "gdsb"):  # the sgn coupling has its exact FP8 form
        with pytest.raises(gsb.GsbError) as e:
            P.run(variant, M=10, R=8, c=0.03, dt=1.0, precision="fx16")
        assert e.value.status == gsb.EUNSUPPORTED
    G = gsb.Problem.dense(I.sk_gauss(64, 1))  # real-valued J has no exact digit form
    with pytest.raises(gsb.GsbError) as e:
        G.run("gbsb", M=10, R=8, c=0.5, dt=1.0, precision="fx16")
    assert e.value.status == gsb.EUNSUPPORTED
