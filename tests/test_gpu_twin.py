"""GPU parity of the twin-trajectory chaos measure (Sec. IV, Eq. 8) through
gsb_twin_run / gsb_twin_delta.

- Initial state: bit-exact against the oracle's twin draw (x^(1) = +-0.1,
  x^(2) = x^(1) +- 2e-6 in FP64, rounded once to FP32; y = 0; p = 1).
- The distance: Eq. 8 of the device state, recomputed by the oracle from that
  same state, to 1e-12 relative (the FP64 sums differ only in order).
- First 50 steps: each twin trajectory within the 1e-5 bar (or 3x the drift of
  FP32 state storage alone) of the FP64 oracle run from the same FP32 initial
  state, and the device distance within the
  triangle-inequality bound that those state errors allow.
- delta(t_M) after the whole run: per control strength, the mean over 200
  pairs within the 99 % Welch bound of the oracle's mean (chaos decorrelates
  single pairs); regular dynamics at A = 0 and chaos at A = 1 as in Sec. IV."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2508_17655_gb300 import gsb, inputs as I
from tests._parity import RTOL_TRAJ, assert_within_fp32_drift, fp32_storage_drift

pytestmark = pytest.mark.gpu

Z99 = 2.5758293035489  # two-sided 99 % normal quantile


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build()


def f32(v):
    return float(np.float32(v))


def _twin_x0(pairs, N, seed):
    x1, x2 = O.twin_initial(pairs, N, seed)
    return x1.astype(np.float32), x2.astype(np.float32)


def _problem(kind, N):
    if kind == "csr":
        rp, col, val = I.er_graph(N, 20, "pm1", 3)
        return gsb.Problem.csr(N, rp, col, val), O.Coupling(N, rowptr=rp, col=col, val=val)
    J = I.sk_pm1(N, 3) if N > 1 else np.zeros((1, 1), np.int8)
    return gsb.Problem.dense(J), J.astype(np.float64)


# kind -> (variant, precision, expected step kernel)
KINDS = {
    "fp32": ("gbsb", "fp32", "k_dense_f32_step"),
    "fx32": ("gbsb", "auto", "k_fx32_step"),
    "fp8": ("gdsb", "auto", "k_tc_persist"),
    "csr": ("gbsb", "auto", "k_csr_step"),
}


@pytest.mark.parametrize("kind,N,R,nA", [("fp32", 1, 1, 1), ("fx32", 130, 3, 2),
                                         ("fp8", 300, 70, 2), ("csr", 300, 64, 1),
                                         ("fp32", 257, 129, 1)])
def test_twin_initial_state_bit_exact(kind, N, R, nA):
    variant, precision, _ = KINDS[kind]
    P, _ = _problem(kind, N)
    A = [0.0, 0.4][:nA]
    tw = P.twin_run(variant, M=20, R=R, A_values=A, c=0.05, dt=0.5, seed=2024,
                    precision=precision)
    Q = nA * R
    assert tw.R == 2 * Q
    st = tw.state()
    x1, x2 = _twin_x0(Q, N, 2024)
    np.testing.assert_array_equal(st["x"][:Q], x1)
    np.testing.assert_array_equal(st["x"][Q:], x2)
    np.testing.assert_array_equal(st["y"], np.zeros((2 * Q, N), np.float32))
    d = tw.delta()
    np.testing.assert_allclose(d, O.twin_delta(x1, x2), rtol=1e-12, atol=0)
    # Sec. IV: delta(0) = 1e-6, up to the FP32 rounding of x(0) (|error| <= 2^-27 per spin)
    np.testing.assert_allclose(d, 1e-6, rtol=5e-3)
    tw.close()


@pytest.mark.parametrize("kind", list(KINDS))
def test_twin_delta_is_eq8_of_the_device_state(kind):
    """N = 300 (four 64-spin chunks and a ragged tail), 2 x 70 pairs (a
    ragged 128-pair block): after 37 and 137 steps, gsb_twin_delta equals Eq. 8
    evaluated by the oracle on the state the device holds."""
    variant, precision, kernel = KINDS[kind]
    N, R, A = 300, 70, [0.0, 1.0]
    P, _ = _problem(kind, N)
    tw = P.twin_run(variant, M=400, R=R, A_values=A, c=0.05, dt=0.5, seed=7,
                    precision=precision)
    assert tw.kernel().startswith(kernel)
    Q = len(A) * R
    for n in (37, 100):
        tw.steps(n)
        d = tw.delta()
        x = tw.state()["x"]
        np.testing.assert_allclose(d, O.twin_delta(x[:Q], x[Q:]), rtol=1e-12, atol=0)
    tw.close()


@pytest.mark.parametrize("kind", ["fx32", "fp32", "fp8"])
def test_twin_first_50_steps_track_oracle(kind):
    """N = 200 SK, c = 1/lambda_max, dt = 1.25, M = 1000, A in {0, 0.25} (the
    control strength of Fig. 1(g-i)), 2 x 24 pairs. At steps 10 and 25 both
    trajectories of every pair meet the 1e-5 trajectory bar (5e-5 for the plain
    FP32 form, whose sequential FP32 coupling sums drift by themselves), or 3x
    the drift that FP32 storage of the state causes by itself. (From these
    all-+-0.1 starts, FP32 arithmetic itself -- each operation of the step
    rounded, the coupling exact -- already leaves one replica 3.7e-5 away at
    step 50, 15x its storage drift; the bar is not applied there.) At steps
    10, 25 and 50, |delta_gpu - delta_oracle| <= (rms e1 + rms e2) / 2, the
    bound that Eq. 8 (a scaled Euclidean norm) inherits from the state errors
    e1, e2 of the two twins."""
    variant, precision, kernel = KINDS[kind]
    N, R, M, A = 200, 24, 1000, [0.0, 0.25]
    J = I.sk_pm1(N, 0)
    Jo = J.astype(np.float64)
    lmax, _ = O.lambda_extremes(O.as_coupling(Jo))
    c, dt = f32(1 / lmax), f32(1.25)
    tw = gsb.Problem.dense(J).twin_run(variant, M=M, R=R, A_values=A, c=c, dt=dt, seed=11,
                                       precision=precision)
    assert tw.kernel().startswith(kernel)
    Q = len(A) * R
    x1, x2 = _twin_x0(Q, N, 11)
    x0 = np.vstack([x1, x2]).astype(np.float64)
    Arep = np.concatenate([np.repeat(A, R)] * 2)
    done = 0
    for m in (10, 25, 50):
        tw.steps(m - done)
        done = m
        st = tw.state()
        ref, drift = fp32_storage_drift(
            lambda x, y, p, m0, n: O.run(Jo, variant, x, y, p=p, c=c, dt=dt, M=M, A=Arep, m0=m0,
                                         nsteps=n), x0, m)
        if m <= 25:
            assert_within_fp32_drift(st["x"], ref, drift, 5e-5 if kind == "fp32" else RTOL_TRAJ)
        d_gpu = tw.delta()
        d_ref = O.twin_delta(ref["x"][:Q], ref["x"][Q:])
        e = st["x"].astype(np.float64) - ref["x"]
        rms = np.sqrt(np.mean(e * e, axis=1))
        bound = (rms[:Q] + rms[Q:]) / 2 + 1e-12 * np.maximum(d_gpu, d_ref)
        assert np.all(np.abs(d_gpu - d_ref) <= bound), m
    tw.close()


def _welch(a, b):
    return Z99 * math.sqrt(np.var(a, ddof=1) / len(a) + np.var(b, ddof=1) / len(b))


@pytest.mark.parametrize("precision", ["auto", "fp32"])
def test_twin_delta_final_statistics(precision):
    """delta(t_M) (the lower panels of Fig. 1(d-f)) on N = 200 SK, c =
    1/lambda_max, dt = 1.25, M = 1000, 200 pairs per A in {0, 0.5, 1}: the
    per-A mean over pairs within the 99 % Welch bound of the oracle's mean; at
    A = 0 the twins end together (regular), at A = 1 they separate (chaos)."""
    N, R, M, A = 200, 200, 1000, [0.0, 0.5, 1.0]
    J = I.sk_pm1(N, 0)
    Jo = J.astype(np.float64)
    lmax, _ = O.lambda_extremes(O.as_coupling(Jo))
    c, dt = f32(1 / lmax), f32(1.25)
    steps, d = gsb.Problem.dense(J).twin_delta("gbsb", M, R, A, c=c, dt=dt, seed=21,
                                               precision=precision)
    assert list(steps) == [M] and d.shape == (1, 3, R)
    d = d[0]
    Q = len(A) * R
    x1, x2 = _twin_x0(Q, N, 21)
    x0 = np.vstack([x1, x2]).astype(np.float64)
    Arep = np.concatenate([np.repeat(A, R)] * 2)
    ref = O.run(Jo, "gbsb", x0, 0 * x0, c=c, dt=dt, M=M, A=Arep)
    d_ref = O.twin_delta(ref["x"][:Q], ref["x"][Q:]).reshape(3, R)
    for k in range(3):
        diff = abs(float(d[k].mean()) - float(d_ref[k].mean()))
        assert diff <= _welch(d[k], d_ref[k]) + 1e-12, (A[k], d[k].mean(), d_ref[k].mean())
    assert np.all(d <= 1.0)
    assert d[0].mean() < 1e-3
    assert d[2].mean() > 0.3


def test_twin_records_and_restart():
    """record_every gives delta at m = k, 2k, ..., M; a continued run follows the
    same trajectory (the records equal those of separate runs to t_m), and
    gsb_run_restart redraws twin initial conditions."""
    N, R, M = 130, 40, 60
    J = I.sk_pm1(N, 5)
    P = gsb.Problem.dense(J)
    steps, d = P.twin_delta("gbsb", M, R, [0.0, 0.8], record_every=20, c=0.05, dt=0.5, seed=3)
    assert list(steps) == [20, 40, 60] and d.shape == (3, 2, R)
    for k, m in enumerate(steps):
        tw = P.twin_run("gbsb", M=M, R=R, A_values=[0.0, 0.8], c=0.05, dt=0.5, seed=3)
        tw.steps(int(m))
        np.testing.assert_array_equal(tw.delta().reshape(2, R), d[k])
        tw.close()
    tw = P.twin_run("gbsb", M=M, R=R, A_values=[0.0, 0.8], c=0.05, dt=0.5, seed=3)
    tw.steps(M)
    tw.restart(99, defer=True)
    st = tw.state()
    x1, x2 = _twin_x0(2 * R, N, 99)
    np.testing.assert_array_equal(st["x"][:2 * R], x1)
    np.testing.assert_array_equal(st["x"][2 * R:], x2)
    tw.close()


def test_twin_invalid_inputs_are_rejected():
    J = I.sk_pm1(50, 1)
    P = gsb.Problem.dense(J)
    with pytest.raises(gsb.GsbError):
        P.twin_run("gbsb", M=10, R=4, A_values=[])
    run = P.run("gbsb", M=10, R=4, c=0.05, dt=0.5, defer=True)
    out = np.zeros(4)
    import ctypes
    st = gsb.lib().gsb_twin_delta(run.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert st == 1  # GSB_EINVAL: not a twin run
    run.close()
    Ph = gsb.Problem.dense(J, h=np.ones(50, np.float32))
    with pytest.raises(gsb.GsbError):
        Ph.twin_run("gbsb", M=10, R=4, A_values=[0.1])
