"""GPU tangent-linear kernel / largest Lyapunov exponent (gsb_lyapunov)
against the FP64 oracle's tangent propagation."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2508_17655_gb300 import gsb, inputs as I
from tests._parity import bf16_split_sum

pytestmark = pytest.mark.gpu

Z99 = 2.5758293035489


def f32(v):
    return float(np.float32(v))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build()


def _oracle_mle(J, variant, R_tot, N, seed, A_rep, c, dt, M, nsteps, renorm, y0_uniform=False,
                x0_range=0.1):
    x0 = O.init_uniform(R_tot, N, seed, rng=x0_range)
    y0 = O.init_uniform(R_tot, N, seed, stream=1, rng=x0_range) if y0_uniform else 0 * x0
    dx0 = O.init_uniform(R_tot, N, seed, stream=4, rng=1.0)
    dx0 /= np.linalg.norm(dx0, axis=1, keepdims=True)
    t = O.tangent_run(J, variant, x0, y0, dx0, c=c, dt=dt, M=M, A=A_rep, nsteps=nsteps,
                      renorm_every=renorm)
    margin = O.run(J, variant, x0, y0, c=c, dt=dt, M=M, A=A_rep, nsteps=nsteps)["margin"]
    return t["log_sum"] / (nsteps * f32(dt)), margin


PRECISIONS = ["fp32", "bf16x3"]
# Decision margin (distance of a wall or sign test from its threshold in the
# oracle's trajectory) below which a replica is excused: a GPU trajectory may
# take the other branch there. FP32 coupling: 2e-6. Split bf16 with the x
# coupling: each step's coupling may differ from the oracle's (on J_hi + J_lo)
# by up to 2^-15 of its magnitude sum_j |J_ij x_j| (x's split residue and the
# dropped J_lo x_lo), of either sign; x moves by c dt^2 times that, and the
# differences build up over the window: 1e-3, the size of the accumulated
# deviation when the per-step ones add like a random walk (not its worst
# case). Its sgn coupling is exact on J_hi + J_lo: the FP32 bar.
NEAR_TIE = {"fp32": 2e-6, "bf16x3": 1e-3}


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("variant", ["gbsb", "bsb", "gdsb", "dsb"])
def test_lyapunov_short_window_matches_oracle(variant, precision):
    """First 50 steps of a 2000-step schedule, renormalised every 10 steps, two
    control strengths x 65 replicas (ragged: three spin tiles, two replica
    tiles of the tensor-core form), SK Gaussian couplings (FP32 J; bf16x3
    splits it): per-replica exponent within 1e-4 (absolute, per unit time) of
    the oracle, replicas with a wall or sign near-tie excused."""
    N, R, M, n, renorm = 300, 65, 2000, 50, 10
    J = I.sk_gauss(N, 7)
    A_vals = [0.1, 0.3]
    c, dt = 0.5, f32(1.25)
    got = gsb.Problem.dense(J).lyapunov(variant, M, R, A_vals, c=c, dt=dt, seed=21,
                                        renorm_every=renorm, nsteps=n, precision=precision)
    A_rep = np.repeat(A_vals, R)
    sign = variant in ("dsb", "gdsb")
    # the split form against the oracle on its own matrix J_hi + J_lo; with the
    # sgn coupling that is exact up to FP32 accumulation (the FP32 bar), with
    # the x coupling the split of x remains (the wider bar)
    Jo = bf16_split_sum(J) if precision == "bf16x3" else J.astype(np.float64)
    want, margin = _oracle_mle(Jo, variant, 2 * R, N, 21, A_rep, c, dt, M, n, renorm)
    ok = margin >= (NEAR_TIE["fp32"] if sign else NEAR_TIE[precision])
    assert ok.mean() > 0.5
    g, w = got.ravel()[ok], want[ok]
    # the inelastic walls can zero a tangent (every oscillator clamped): -inf on both sides
    both_inf = np.isneginf(g) & np.isneginf(w)
    err = np.abs(g[~both_inf] - w[~both_inf])
    assert not np.isnan(g).any() and not np.isnan(w).any()
    assert np.array_equal(np.isneginf(g), np.isneginf(w))
    assert err.size == 0 or np.all(err <= 1e-4), f"max |mle gpu - oracle| {err.max():.2e}"


@pytest.mark.parametrize("precision", PRECISIONS)
def test_lyapunov_config5_shape_sampled(precision):
    """The chaos configuration as the bench runs it (N = 2000 SK Gaussian,
    16 control strengths x 256 replicas in one call, c = 0.5, dt = 1.25,
    M = 2000, renormalised every 10 steps), first 50 steps: 16 sampled replicas
    (one per control strength) within 1e-4 of the oracle's exponent."""
    N, R, M, n, renorm = 2000, 256, 2000, 50, 10
    A16 = [0.025 * k for k in range(16)]
    J = I.sk_gauss(N, 0)
    c, dt = 0.5, f32(1.25)
    got = gsb.Problem.dense(J).lyapunov("gbsb", M, R, A16, c=c, dt=dt, seed=3,
                                        renorm_every=renorm, nsteps=n,
                                        precision=precision).ravel()
    pick = np.array([k * R + (37 * k) % R for k in range(16)])
    x0 = O.init_uniform(16 * R, N, 3)[pick]
    dx0 = O.init_uniform(16 * R, N, 3, stream=4, rng=1.0)[pick]
    dx0 /= np.linalg.norm(dx0, axis=1, keepdims=True)
    A_rep = np.repeat(A16, R)[pick]
    Jo = J.astype(np.float64)
    t = O.tangent_run(Jo, "gbsb", x0, 0 * x0, dx0, c=c, dt=dt, M=M, A=A_rep, nsteps=n,
                      renorm_every=renorm)
    want = t["log_sum"] / (n * dt)
    margin = O.run(Jo, "gbsb", x0, 0 * x0, c=c, dt=dt, M=M, A=A_rep, nsteps=n)["margin"]
    ok = margin >= NEAR_TIE[precision]
    assert ok.sum() >= 10
    err = np.abs(got[pick] - want)[ok]
    assert np.all(err <= 1e-4), f"max |mle gpu - oracle| {err.max():.2e}"


@pytest.mark.parametrize("precision", PRECISIONS)
def test_lyapunov_unstable_equilibrium_growth_rate(precision):
    """Near the x = 0 equilibrium of a ferromagnet (J = 1 - I) with p ~ 1, the
    uniform mode grows by mu per step, mu^2 - (2 - k dt^2) mu + 1 = 0,
    k = p - c (N - 1): GPU exponent equals the oracle's and approaches ln(mu)/dt."""
    N, R, M, n = 64, 16, 10 ** 6, 400
    J = (-I.complete(N)).astype(np.float32)
    c, dt = f32(0.02), f32(0.3)
    got = gsb.Problem.dense(J, validate=True).lyapunov("bsb", M, R, [0.0], c=c, dt=dt, seed=3,
                                                       renorm_every=10, nsteps=n,
                                                       x0_range=1e-30, precision=precision)[0]
    want, _ = _oracle_mle(J.astype(np.float64), "bsb", R, N, 3, np.zeros(R), c, dt, M, n, 10,
                          x0_range=1e-30)
    np.testing.assert_allclose(got, want, rtol=1e-4)
    k = 1.0 - c * (N - 1)
    b = 2 - k * dt * dt
    mu = (b + math.sqrt(b * b - 4)) / 2
    # a random start vector overlaps the growing mode by ~N^-1/2: the finite-time
    # estimate sits below ln(mu)/dt by about ln(overlap)/(n dt) (up to ~12 % here);
    # the oracle pins the rate itself with an aligned start vector
    rate = math.log(mu) / dt
    assert np.all(got <= rate * 1.01) and np.all(got >= rate * 0.88)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("variant", ["gbsb", "gdsb"])
def test_lyapunov_long_window_statistics(variant, precision):
    """The first 300 steps of 600-step runs (long enough for the trajectories
    to decorrelate, before the end of the schedule pins every oscillator to a
    wall and zeroes every tangent), 4 control strengths x 64 replicas: mean
    exponent per strength within the 99 % Welch bound of the oracle's."""
    N, R, M, n = 200, 64, 600, 300
    J = I.sk_gauss(N, 9)
    A_vals = [0.0, 0.2, 0.4, 0.6]
    c, dt = 0.5, f32(1.0)
    got = gsb.Problem.dense(J).lyapunov(variant, M, R, A_vals, c=c, dt=dt, seed=5, renorm_every=10,
                                        nsteps=n, precision=precision)
    want, _ = _oracle_mle(J.astype(np.float64), variant, 4 * R, N, 5, np.repeat(A_vals, R), c, dt,
                          M, n, 10)
    want = want.reshape(4, R)
    assert not np.isnan(got).any() and not np.isnan(want).any()
    for k in range(4):
        g, w = got[k], want[k]
        # a tangent zeroed by the walls (all oscillators clamped) gives -inf
        gi, wi = np.isneginf(g).mean(), np.isneginf(w).mean()
        assert abs(gi - wi) <= 0.2, (A_vals[k], gi, wi)
        g, w = g[np.isfinite(g)], w[np.isfinite(w)]
        if len(g) < 8 or len(w) < 8:
            continue
        bound = Z99 * math.sqrt(np.var(g, ddof=1) / len(g) + np.var(w, ddof=1) / len(w)) + 1e-6
        assert abs(g.mean() - w.mean()) <= bound, (A_vals[k], g.mean(), w.mean(), bound)


def test_lyapunov_bf16x3_agrees_with_fp32_and_rejects_other_forms():
    """The two coupling forms on the same runs (N = 257: a ragged third spin
    tile; 3 x 50 replicas), 40 steps: exponents within 1e-4 of each other
    wherever the oracle's trajectory has no near-tie decision (margin 1e-3, as
    for the split form above); a form the tangent path does not have is
    refused."""
    N, R, M, n = 257, 50, 1000, 40
    J = I.sk_gauss(N, 4)
    A_vals = [0.0, 0.2, 0.4]
    P = gsb.Problem.dense(J)
    kw = dict(c=0.5, dt=f32(1.25), seed=8, renorm_every=10, nsteps=n)
    a = P.lyapunov("gbsb", M, R, A_vals, precision="fp32", **kw).ravel()
    b = P.lyapunov("gbsb", M, R, A_vals, precision="bf16x3", **kw).ravel()
    x0 = O.init_uniform(3 * R, N, 8)
    margin = O.run(J.astype(np.float64), "gbsb", x0, 0 * x0, c=0.5, dt=f32(1.25), M=M,
                   A=np.repeat(A_vals, R), nsteps=n)["margin"]
    ok = margin >= NEAR_TIE["bf16x3"]
    assert ok.mean() > 0.5
    a, b = a[ok], b[ok]
    assert np.array_equal(np.isneginf(a), np.isneginf(b))
    fin = np.isfinite(a)
    assert np.max(np.abs(a[fin] - b[fin])) <= 1e-4
    with pytest.raises(gsb.GsbError) as e:
        P.lyapunov("gbsb", M, R, [0.0], precision="fp8", **kw)
    assert e.value.status == gsb.EUNSUPPORTED


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("N", [1, 2, 129])
def test_lyapunov_degenerate_and_edge_sizes(N, precision):
    """N = 1 (no coupling at all), N = 2 and N = 129 (one spin past a tile),
    3 replicas, 30 steps: the exponents match the oracle's within 1e-4 (the
    split form against the oracle on J_hi + J_lo), replicas with a near-tie
    decision excused."""
    J = I.sk_gauss(N, 3) if N > 1 else np.zeros((1, 1), np.float32)
    R, M, n = 3, 500, 30
    c, dt = 0.5, f32(0.9)
    got = gsb.Problem.dense(J).lyapunov("gbsb", M, R, [0.2], c=c, dt=dt, seed=5, renorm_every=10,
                                        nsteps=n, precision=precision).ravel()
    Jo = bf16_split_sum(J) if precision == "bf16x3" else J.astype(np.float64)
    want, margin = _oracle_mle(Jo, "gbsb", R, N, 5, np.full(R, 0.2), c, dt, M, n, 10)
    ok = margin >= NEAR_TIE[precision]
    assert np.array_equal(np.isneginf(got[ok]), np.isneginf(want[ok]))
    fin = ok & np.isfinite(want)
    assert np.all(np.abs(got[fin] - want[fin]) <= 1e-4), (got, want)
