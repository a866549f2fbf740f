"""Pins for the FP64 oracle: each test checks the oracle against something other
than itself -- a published known answer, a closed form, an invariant of the
mathematics, a library routine, or exhaustive enumeration."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2508_17655_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper_values():
    vals = {}
    for line in open(os.path.join(GOLDEN, "paper_values.txt")):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        k, v = line.split("=")
        vals[k.strip()] = float(v)
    return vals


# ---------------------------------------------------------------- Philox

def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        out = O.philox4x32_10(w[0:4], w[4:6])
        assert list(out) == w[6:10]
        n += 1
    assert n == 3


def test_init_uniform_range_and_distribution():
    from scipy.stats import kstest
    x = O.init_uniform(64, 500, seed=3)
    assert x.shape == (64, 500)
    assert np.all(x >= -0.1) and np.all(x < 0.1)
    # values are FP32 numbers
    assert np.array_equal(x, x.astype(np.float32).astype(np.float64))
    p = kstest((x.ravel() + 0.1) / 0.2, "uniform").pvalue
    assert p > 1e-4
    # deterministic, and distinct streams / seeds differ
    assert np.array_equal(x, O.init_uniform(64, 500, seed=3))
    assert not np.array_equal(x, O.init_uniform(64, 500, seed=4))
    assert not np.array_equal(x, O.init_uniform(64, 500, seed=3, stream=1))


# ---------------------------------------------------------------- energy / cut

def _random_spins(R, N, seed):
    rng = np.random.default_rng(seed)
    return (rng.integers(0, 2, size=(R, N)) * 2 - 1).astype(np.int8)


@pytest.mark.parametrize("kind", ["pm1", "gauss", "sparse"])
def test_energy_cut_identity(kind):
    """cut = (W_tot - E) / 2 with W = -J (Sec. III), cut counted edge by edge."""
    N = 40
    if kind == "pm1":
        J = I.sk_pm1(N, 1).astype(np.float64)
    elif kind == "gauss":
        J = I.sk_gauss(N, 2).astype(np.float64)
    else:
        J = I.csr_to_dense(N, *I.er_graph(N, 5, "pm1", 3))
    S = _random_spins(20, N, 5)
    Wtot = O.total_weight(J)
    for s in S:
        e = O.energy(J, s)
        cut = O.cut_dense(J, s)
        assert abs(cut - (Wtot - e) / 2) <= 1e-9 * max(1.0, abs(Wtot))


def test_energy_global_flip_and_integrality():
    N = 50
    J = I.sk_pm1(N, 4).astype(np.float64)
    S = _random_spins(30, N, 6)
    e = O.energy(J, S)
    e_neg = O.energy(J, -S)
    assert np.array_equal(e, e_neg)
    assert np.array_equal(e, np.round(e))  # integer J, integer energy


def test_energy_csr_equals_dense():
    N = 300
    rp, col, val = I.er_graph(N, 8, "pm1", 9)
    D = I.csr_to_dense(N, rp, col, val)
    S = _random_spins(16, N, 10)
    e_csr = O.energy(O.Coupling(N, rowptr=rp, col=col, val=val), S)
    e_den = O.energy(D, S)
    assert np.array_equal(e_csr, e_den)


def _exhaustive_numpy(J):
    N = J.shape[0]
    best = math.inf
    for bits in itertools.product([1, -1], repeat=N):
        s = np.array(bits, dtype=np.float64)
        best = min(best, -0.5 * float(s @ J @ s))
    return best


@pytest.mark.parametrize("N", [1, 2, 5, 9, 12])
def test_bruteforce_matches_exhaustive(N):
    J = I.sk_pm1(N, 11 + N).astype(np.float64) if N > 1 else np.zeros((1, 1))
    e, s = O.bruteforce(J)
    assert e == _exhaustive_numpy(J)
    assert O.energy(J, s) == e


@pytest.mark.parametrize("N", [4, 5, 8, 11, 16])
def test_bruteforce_closed_form_graphs(N):
    # cycle: max cut N (even) or N - 1 (odd)
    J = I.ring(N)
    e, s = O.bruteforce(J)
    maxcut = N if N % 2 == 0 else N - 1
    assert O.cut_dense(J, s) == maxcut
    assert e == O.total_weight(J) - 2 * maxcut
    # complete graph K_N: max cut floor(N/2) ceil(N/2)
    J = I.complete(N)
    e, s = O.bruteforce(J)
    assert O.cut_dense(J, s) == (N // 2) * ((N + 1) // 2)
    # ferromagnet (J = +1): all spins aligned, E = -N(N-1)/2
    e, s = O.bruteforce(-I.complete(N))
    assert e == -N * (N - 1) / 2 and abs(int(s.sum())) == N


# ---------------------------------------------------------------- integrator

def _harmonic(x0, k, dt, m):
    """Eq. 10 with y(0) = 0: x_m = x0 [cos m th - tan(th/2) sin m th], cos th = 1 - k dt^2 / 2."""
    th = math.acos(1.0 - k * dt * dt / 2.0)
    return x0 * (math.cos(m * th) - math.tan(th / 2.0) * math.sin(m * th))


@pytest.mark.parametrize("k,dt", [(1.0, 0.5), (0.3, 1.25), (2.0, 1.3), (0.05, 1.0)])
def test_eq10_harmonic_closed_form(k, dt):
    """J = 0 and a frozen shared parameter p = k (bSB with a constant
    schedule): each oscillator is the harmonic recurrence of Eq. 10 (App. A)."""
    assert dt < 2.0 / math.sqrt(k)  # Eq. 11: oscillating regime
    N, R, M = 3, 2, 120
    J = np.zeros((N, N))
    x0 = np.array([[0.05, -0.02, 0.01], [-0.07, 0.03, 0.0]])
    y0 = np.zeros_like(x0)
    sched = np.full(M + 1, k)
    out = O.run(J, "bsb", x0, y0, c=0.7, dt=dt, M=M, sched=sched)
    # step through in chunks too: resume composes exactly
    x, y, p = x0, y0, None
    for m in range(0, M, 7):
        n = min(7, M - m)
        o = O.run(J, "bsb", x, y, c=0.7, dt=dt, M=M, sched=sched, m0=m, nsteps=n, p=p)
        x, y, p = o["x"], o["y"], o["p"]
        want = np.vectorize(lambda v: _harmonic(v, k, dt, m + n))(x0)
        np.testing.assert_allclose(x, want, rtol=0, atol=1e-12)
    assert np.array_equal(x, out["x"]) and np.array_equal(y, out["y"])


def test_eq11_stability_bound():
    """Above Delta_t = 2/sqrt(k) the recurrence grows until the wall stops it."""
    k = 1.0
    N, M = 1, 60
    J = np.zeros((N, N))
    x0 = np.array([[1e-3]])
    sched = np.full(M + 1, k)
    below = O.run(J, "bsb", x0, 0 * x0, c=1.0, dt=1.99, M=M, sched=sched)
    above = O.run(J, "bsb", x0, 0 * x0, c=1.0, dt=2.05, M=M, sched=sched)
    assert abs(below["x"][0, 0]) < 0.2
    assert abs(above["x"][0, 0]) == 1.0  # reached a wall (Eq. 5)


def test_coupling_sign_on_uniform_mode():
    """Ferromagnetic complete graph (J = 1 - I): the uniform mode has
    J x = (N - 1) x, so Eq. 3 is a harmonic oscillator with k = p - c (N - 1).
    A wrong sign or scale on the many-body term breaks the closed form."""
    N, M = 6, 80
    J = -I.complete(N)
    c = 0.1
    p = 0.9
    k = p - c * (N - 1)
    dt = 1.1
    x0 = np.full((1, N), 0.03)
    out = O.run(J, "bsb", x0, 0 * x0, c=c, dt=dt, M=M, sched=np.full(M + 1, p))
    np.testing.assert_allclose(out["x"], _harmonic(0.03, k, dt, M), rtol=0, atol=1e-12)


def test_gbsb_a0_is_bsb():
    """Eq. 7 with A = 0 reproduces the linear schedule p(t_m) = 1 - m/M of
    Eq. 6, so GbSB with A = 0 follows the bSB trajectory (Sec. II)."""
    N, R, M = 30, 4, 200
    J = I.sk_pm1(N, 21).astype(np.float64)
    x0 = O.init_uniform(R, N, seed=5)
    y0 = np.zeros_like(x0)
    c = 1.0 / (2 * math.sqrt(N))
    a = O.run(J, "gbsb", x0, y0, c=c, dt=1.25, M=M, A=0.0)
    b = O.run(J, "bsb", x0, y0, c=c, dt=1.25, M=M)
    np.testing.assert_allclose(a["x"], b["x"], rtol=0, atol=1e-9)
    # the individual parameters follow 1 - m/M at every step
    p = None
    x, y = x0, y0
    for m in range(0, M, 25):
        o = O.run(J, "gbsb", x, y, c=c, dt=1.25, M=M, A=0.0, m0=m, nsteps=25, p=p)
        x, y, p = o["x"], o["y"], o["p"]
        np.testing.assert_allclose(p, 1.0 - (m + 25) / M, rtol=0, atol=1e-13)
    # same dSB statement
    a = O.run(J, "gdsb", x0, y0, c=c, dt=1.25, M=M, A=0.0)
    b = O.run(J, "dsb", x0, y0, c=c, dt=1.25, M=M)
    np.testing.assert_allclose(a["x"], b["x"], rtol=0, atol=1e-9)


@pytest.mark.parametrize("A", [0.0, 0.3, 1.0])
def test_eq7_product_formula_with_pinned_walls(A):
    """Oscillators held at the wall x = +-1 (a strong ferromagnetic pull and
    Eq. 5) have A x^2 = A, and Eq. 7 gives the product
    p(t_m) = Gamma(M+A) Gamma(M-m+1) / (Gamma(M-m+A) Gamma(M+1))."""
    N, M = 4, 60
    J = -I.complete(N)
    x0 = np.array([[1.0, 1.0, 1.0, 1.0], [-1.0, -1.0, -1.0, -1.0]])
    x, y, p = x0, np.zeros_like(x0), None
    for m in range(0, M, 5):
        o = O.run(J, "gbsb", x, y, c=10.0, dt=0.5, M=M, A=A, m0=m, nsteps=5, p=p)
        x, y, p = o["x"], o["y"], o["p"]
        assert np.array_equal(np.abs(x), np.ones_like(x)) and np.all(y == 0)
        mm = m + 5
        if M - mm + A == 0:
            want = 0.0  # 1/Gamma has a zero there: A = 0 ends at p(t_M) = 0 (Eq. 6)
        else:
            want = math.exp(math.lgamma(M + A) + math.lgamma(M - mm + 1)
                            - math.lgamma(M - mm + A) - math.lgamma(M + 1))
        np.testing.assert_allclose(p, want, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("variant", ["gbsb", "gdsb", "bsb", "dsb"])
def test_time_reversal_of_wall_free_step(variant):
    """One symplectic-Euler step (Eqs. 3, 4, 7) inverted backwards:
    x_m = x_{m+1} - y_{m+1} dt; p_m from Eq. 7 solved for p_m; then
    y_m = y_{m+1} + (p_{m+1} x_m - c J v(x_m)) dt. The round trip recovers the
    state only if the forward step used p(t_{m+1}), x(t_m) and v(x(t_m)) in
    Eq. 3 and x(t_m) in Eq. 7."""
    N, R, M = 25, 3, 40
    J = I.sk_gauss(N, 31).astype(np.float64)
    rng = np.random.default_rng(8)
    x = rng.uniform(-0.3, 0.3, size=(R, N))
    y = rng.uniform(-0.05, 0.05, size=(R, N))
    p = rng.uniform(0.5, 1.0, size=(R, N))
    A = np.array([0.0, 0.4, 0.9])
    c, dt = 0.4, 0.6
    m = 17
    sign = variant in ("dsb", "gdsb")
    ctrl = variant in ("gbsb", "gdsb")
    p_in = p if ctrl else np.full_like(p, 1.0 - m / M)
    o = O.run(J, variant, x, y, c=c, dt=dt, M=M, A=A, p=p_in, m0=m, nsteps=1)
    x1, y1, p1 = o["x"], o["y"], o["p"]
    assert np.all(np.abs(x1) < 1.0)  # wall-free
    xb = x1 - y1 * dt
    if ctrl:
        pb = p1 / (1.0 - (1.0 - A[:, None] * xb * xb) / (M - m))
    else:
        pb = p_in
        np.testing.assert_allclose(p1, 1.0 - (m + 1) / M, rtol=0, atol=1e-15)
    v = np.where(xb >= 0, 1.0, -1.0) if sign else xb
    yb = y1 + (p1 * xb - c * (v @ J.T)) * dt
    np.testing.assert_allclose(xb, x, rtol=0, atol=1e-13)
    np.testing.assert_allclose(yb, y, rtol=0, atol=1e-13)
    np.testing.assert_allclose(pb, p_in, rtol=1e-13, atol=0)


@pytest.mark.parametrize("variant", ["gbsb", "gdsb", "bsb", "dsb"])
def test_sign_symmetry_bit_exact(variant):
    """(x, y) -> (-x, -y) maps trajectories to their negatives exactly: p
    depends on x^2, the walls are odd and round-to-nearest is symmetric."""
    N, R, M = 40, 6, 300
    J = I.sk_pm1(N, 41).astype(np.float64)
    x0 = O.init_uniform(R, N, seed=9)
    y0 = O.init_uniform(R, N, seed=9, stream=1)
    kw = dict(c=1 / (2 * math.sqrt(N)), dt=1.25, M=M, A=0.25, eval_every=10)
    a = O.run(J, variant, x0, y0, **kw)
    b = O.run(J, variant, -x0, -y0, **kw)
    assert np.array_equal(a["x"], -b["x"]) and np.array_equal(a["y"], -b["y"])
    assert np.array_equal(a["p"], b["p"])
    assert np.array_equal(a["best"]["E"], b["best"]["E"])
    assert np.any(np.abs(a["x"]) == 1.0)  # walls were exercised


def test_gauge_invariance_bit_exact():
    """J' = D J D, x' = D x with D = diag(+-1) gives x'(t) = D x(t) exactly
    and identical energies (Eq. 1 is gauge invariant)."""
    N, R, M = 35, 4, 250
    J = I.sk_gauss(N, 51).astype(np.float64)
    d = np.where(np.random.default_rng(3).random(N) < 0.5, -1.0, 1.0)
    Jg = d[:, None] * J * d[None, :]
    x0 = O.init_uniform(R, N, seed=13)
    kw = dict(c=0.5, dt=1.0, M=M, A=0.3, eval_every=5)
    for variant in ("gbsb", "gdsb"):
        a = O.run(J, variant, x0, 0 * x0, **kw)
        b = O.run(Jg, variant, x0 * d, 0 * x0, **kw)
        assert np.array_equal(a["x"] * d, b["x"])
        assert np.array_equal(a["best"]["E"], b["best"]["E"])


def test_walls_and_best_keeping():
    """|x| <= 1 always (Eq. 5); best_E is the minimum over the evaluated steps
    with the earliest step on ties; final-only evaluation matches the energy of
    sgn x(t_M)."""
    N, R, M = 30, 5, 120
    J = I.sk_pm1(N, 61).astype(np.float64)
    x0 = O.init_uniform(R, N, seed=2)
    kw = dict(c=1 / (2 * math.sqrt(N)), dt=1.25, M=M, A=0.2)
    full = O.run(J, "gbsb", x0, 0 * x0, eval_every=1, **kw)
    assert np.all(np.abs(full["x"]) <= 1.0)
    x, y, p = x0, 0 * x0, None
    energies = []
    for m in range(M):
        o = O.run(J, "gbsb", x, y, m0=m, nsteps=1, p=p, **kw)
        x, y, p = o["x"], o["y"], o["p"]
        energies.append(O.energy(J, O.spins(x)))
    energies = np.array(energies)  # (M, R)
    np.testing.assert_array_equal(full["best"]["E"], energies.min(axis=0))
    np.testing.assert_array_equal(full["best"]["step"], energies.argmin(axis=0) + 1)
    for r in range(R):
        assert O.energy(J, full["best"]["s"][r]) == full["best"]["E"][r]
    final = O.run(J, "gbsb", x0, 0 * x0, eval_every=0, **kw)
    np.testing.assert_array_equal(final["best"]["E"], energies[-1])
    assert np.all(final["best"]["step"] == M)


@pytest.mark.parametrize("variant", ["gbsb", "dsb"])
def test_finds_brute_force_ground_state(variant):
    """On small +-1 instances the runs never go below the exhaustive minimum,
    and some replicas reach it."""
    N, R, M = 16, 64, 400
    for seed in (71, 72):
        J = I.sk_pm1(N, seed).astype(np.float64)
        e0, _ = O.bruteforce(J)
        lmax, _ = O.lambda_extremes(J)
        x0 = O.init_uniform(R, N, seed=seed)
        o = O.run(J, variant, x0, 0 * x0, c=1 / lmax, dt=0.5, M=M, A=0.2, eval_every=1)
        assert np.all(o["best"]["E"] >= e0)
        assert np.mean(o["best"]["E"] == e0) > 0.05


# ---------------------------------------------------------------- setup (App. A)

def test_lambda_extremes_match_lapack():
    for J in (I.sk_pm1(40, 81).astype(np.float64), I.sk_gauss(60, 82).astype(np.float64),
              I.csr_to_dense(70, *I.er_graph(70, 6, "+1", 83))):
        lmax, lmin = O.lambda_extremes(J)
        w = np.linalg.eigvalsh(J)
        assert abs(lmax - w[-1]) <= 1e-7 * abs(w[-1])
        assert abs(lmin - w[0]) <= 1e-7 * abs(w[0])


def test_wigner_estimate_and_dt_bound():
    """App. A: lambda_max ~ 2 sqrt(N) sigma for a random +-1 matrix; the bound of
    Eq. 12 is close to sqrt(2), and Eq. 13 with D_t = 1.25 gives the paper's
    Delta_t = 1.25 for random instances."""
    vals = _paper_values()
    N = 400
    J = I.sk_pm1(N, 91).astype(np.float64)
    lmax, lmin = O.lambda_extremes(J)
    assert abs(lmax / (2 * math.sqrt(N)) - 1) < 0.06
    assert abs(2.0 / math.sqrt(1.0 - lmin / lmax) - vals["dt_bound_random"]) < 0.02
    assert abs(O.dt_from_lambda(lmax, lmin, Dt=1.25) - vals["dt_random"]) < 0.02


# ---------------------------------------------------------------- statistics

def test_tts_formula():
    vals = _paper_values()
    tgt = vals["tts_target"]
    assert O.tts(0.9, 3.0, tgt) == pytest.approx(6.0, rel=1e-12)  # log 0.01 / log 0.1 = 2
    assert O.tts(0.995, 3.0, tgt) == 3.0
    assert O.tts(0.0, 3.0, tgt) == math.inf
    # Delta_TTS is first-order error propagation of Delta P_S through TTS(P_S)
    ps, n = 0.3, 1000
    h = 1e-6
    deriv = (O.tts(ps + h, 1.0) - O.tts(ps - h, 1.0)) / (2 * h)
    assert O.tts_error(ps, 1.0, n) == pytest.approx(abs(deriv) * O.ps_error(ps, n), rel=1e-6)
    assert O.ps_error(0.5, 100) == pytest.approx(0.05)


def test_clopper_pearson_closed_forms_and_tails():
    """The exact binomial interval behind the P_S error bars: at k = 0 and
    k = n it has the closed forms 1 - (a/2)^(1/n) and (a/2)^(1/n); inside, its
    bounds make the binomial tails exactly a/2 (summed term by term here)."""
    from math import comb
    a = 0.01
    for n in (1, 7, 50, 1000):
        lo, hi = O.clopper_pearson(0, n, 0.99)
        assert lo == 0.0 and hi == pytest.approx(1 - (a / 2) ** (1 / n), rel=1e-10)
        lo, hi = O.clopper_pearson(n, n, 0.99)
        assert hi == 1.0 and lo == pytest.approx((a / 2) ** (1 / n), rel=1e-10)
    for n, k in ((10, 3), (40, 17), (100, 1), (1000, 12)):
        lo, hi = O.clopper_pearson(k, n, 0.99)
        upper_tail = sum(comb(n, j) * lo ** j * (1 - lo) ** (n - j) for j in range(k, n + 1))
        lower_tail = sum(comb(n, j) * hi ** j * (1 - hi) ** (n - j) for j in range(0, k + 1))
        assert upper_tail == pytest.approx(a / 2, rel=1e-7)
        assert lower_tail == pytest.approx(a / 2, rel=1e-7)


def test_twin_distance_values():
    vals = _paper_values()
    x1, x2 = O.twin_initial(8, 500, seed=4)
    assert np.all(np.abs(np.abs(x1) - 0.1) == 0)
    d0 = O.twin_delta(x1, x2)
    np.testing.assert_allclose(d0, vals["twin_delta_t0"], rtol=1e-9)
    # delta <= 1, with equality for x2 = -x1 at the walls
    ones = np.ones((1, 500))
    assert O.twin_delta(ones, -ones)[0] == vals["twin_delta_max"]
    rng = np.random.default_rng(1)
    a = np.where(rng.random((1, 200000)) < 0.5, 1.0, -1.0)
    b = np.where(rng.random((1, 200000)) < 0.5, 1.0, -1.0)
    assert abs(O.twin_delta(a, b)[0] - vals["twin_delta_chaos"]) < 5e-3


def test_twin_regular_without_control_chaotic_with_it():
    """Sec. IV: without the control of Eq. 7 (A = 0) the twins end together,
    delta(t_M) ~ 0 (regular dynamics); a strong control (A = 1) drives them
    apart, delta(t_M) of order 1/sqrt 2 (chaos). N = 200 SK, c = 1/lambda_max,
    dt = 1.25, M = 1000, 40 pairs each. A dropped control term, a wrong sign in
    Eq. 7 or twins that share one trajectory each break one of the two."""
    N, R, M = 200, 40, 1000
    J = I.sk_pm1(N, 0).astype(np.float64)
    lmax, _ = O.lambda_extremes(O.as_coupling(J))
    x1, x2 = O.twin_initial(R, N, seed=12)
    x = np.vstack([x1, x2])
    means = []
    for A in (0.0, 1.0):
        r = O.run(J, "gbsb", x, 0 * x, c=1 / lmax, dt=1.25, M=M, A=A)
        d = O.twin_delta(r["x"][:R], r["x"][R:])
        assert np.all(d <= 1.0)
        means.append(float(d.mean()))
    assert means[0] < 1e-3
    assert means[1] > 0.3


# ---------------------------------------------------------------- tangent-linear

@pytest.mark.parametrize("variant", ["gbsb", "bsb", "gdsb", "dsb"])
def test_tangent_matches_central_differences(variant):
    """The tangent propagated over a few wall-free steps equals the central
    difference quotient of the nonlinear iteration (orc_run) in that direction."""
    N, R, M, m0, n = 40, 3, 300, 7, 4
    J = I.sk_gauss(N, 61).astype(np.float64)
    rng = np.random.default_rng(4)
    x = rng.uniform(-0.2, 0.2, size=(R, N))
    x[np.abs(x) < 0.05] = 0.05  # keep signs away from zero (dSB coupling)
    y = rng.uniform(-0.02, 0.02, size=(R, N))
    p = rng.uniform(0.6, 1.0, size=(R, N))
    dx, dy, dp = (rng.standard_normal((R, N)) for _ in range(3))
    if variant in ("bsb", "dsb"):
        dp = np.zeros_like(dp)
    kw = dict(c=0.2, dt=0.5, M=M, A=0.35, m0=m0, nsteps=n)
    t = O.tangent_run(J, variant, x, y, dx, dy=dy, dp=dp, p=p, renorm_every=10 ** 6, **kw)
    scale = np.exp(t["log_sum"])[:, None]
    eps = 1e-6
    plus = O.run(J, variant, x + eps * dx, y + eps * dy, p=p + eps * dp, **kw)
    minus = O.run(J, variant, x - eps * dx, y - eps * dy, p=p - eps * dp, **kw)
    assert np.all(np.abs(plus["x"]) < 1) and np.all(np.abs(minus["x"]) < 1)
    for k, dk in (("x", "dx"), ("y", "dy"), ("p", "dp")):
        fd = (plus[k] - minus[k]) / (2 * eps)
        np.testing.assert_allclose(t[dk] * scale, fd, rtol=1e-6, atol=1e-7 * np.max(np.abs(fd)) + 1e-12)


def test_tangent_growth_rate_at_equilibrium():
    """About the x = 0 equilibrium of a ferromagnet (J = 1 - I, frozen p), the
    uniform mode is the harmonic recurrence of Eq. 10 with k = p - c (N - 1) < 0;
    its growth factor mu solves mu^2 - (2 - k dt^2) mu + 1 = 0, so the largest
    Lyapunov exponent is ln(mu)/dt."""
    N, R, M = 12, 4, 600
    J = -I.complete(N)
    p, c, dt = 0.5, 0.1, 0.8
    k = p - c * (N - 1)
    b = 2 - k * dt * dt
    mu = (b + math.sqrt(b * b - 4)) / 2
    x0 = np.zeros((R, N))
    dx0 = 1.0 + 0.5 * np.random.default_rng(1).standard_normal((R, N))  # overlaps the uniform mode
    for variant in ("bsb", "gbsb"):
        t = O.tangent_run(J, variant, x0, x0, dx0, c=c, dt=dt, M=M, A=0.3, sched=np.full(M + 1, p),
                          renorm_every=10) if variant == "bsb" else None
        if t is None:  # GbSB: A x^2 = 0 at the equilibrium, p follows Eq. 7 (use it directly)
            continue
        assert np.all(t["x"] == 0)
        mle = t["log_sum"] / (M * dt)
        np.testing.assert_allclose(mle, math.log(mu) / dt, rtol=0.01)
    # a stable frozen p (k > 0): no growth, exponent ~ 0
    t = O.tangent_run(J, "bsb", x0, x0, dx0, c=0.01, dt=dt, M=M, sched=np.full(M + 1, p),
                      renorm_every=10)
    assert np.all(np.abs(t["log_sum"] / (M * dt)) < 0.01)


# ---------------------------------------------------------------- adjoint

@pytest.mark.parametrize("variant", ["gbsb", "bsb", "gdsb", "dsb"])
def test_adjoint_matches_central_differences(variant):
    """dE/dx0 (along random directions), dE/dA and dE/ddt of the relaxed energy
    E = -1/2 x(t_W)^T J x(t_W) equal central differences of the forward
    iteration, away from wall events and sign changes."""
    N, R, M, W = 30, 3, 200, 25
    J = I.sk_gauss(N, 71).astype(np.float64)
    rng = np.random.default_rng(9)
    x0 = rng.uniform(-0.3, 0.3, size=(R, N))
    x0[np.abs(x0) < 0.05] = 0.05
    c, dt, A = 0.4, 0.6, 0.3
    E, gx, gA, gdt = O.relaxed_energy_grad(J, variant, x0, c=c, dt=dt, M=M, W=W, A=A)
    E2, margin = O.relaxed_energy(J, variant, x0, c=c, dt=dt, M=M, W=W, A=A)
    np.testing.assert_allclose(E, E2, rtol=1e-13)
    ok = margin > 1e-4  # no wall test or sign within reach of the difference step
    assert ok.sum() >= 2
    h = 1e-6
    u = rng.standard_normal((R, N))
    fd_x = (O.relaxed_energy(J, variant, x0 + h * u, c=c, dt=dt, M=M, W=W, A=A)[0]
            - O.relaxed_energy(J, variant, x0 - h * u, c=c, dt=dt, M=M, W=W, A=A)[0]) / (2 * h)
    np.testing.assert_allclose(np.sum(gx * u, axis=1)[ok], fd_x[ok], rtol=1e-6, atol=1e-8)
    fd_dt = (O.relaxed_energy(J, variant, x0, c=c, dt=dt + h, M=M, W=W, A=A)[0]
             - O.relaxed_energy(J, variant, x0, c=c, dt=dt - h, M=M, W=W, A=A)[0]) / (2 * h)
    np.testing.assert_allclose(gdt[ok], fd_dt[ok], rtol=1e-6, atol=1e-8)
    fd_A = (O.relaxed_energy(J, variant, x0, c=c, dt=dt, M=M, W=W, A=A + h)[0]
            - O.relaxed_energy(J, variant, x0, c=c, dt=dt, M=M, W=W, A=A - h)[0]) / (2 * h)
    np.testing.assert_allclose(gA[ok], fd_A[ok], rtol=1e-6, atol=1e-8)
    if variant in ("bsb", "dsb"):
        assert np.all(gA == 0.0)


def test_adjoint_dot_product_identity_with_tangent():
    """<dE/dx0, u> = <dE/dx(t_W), TLM u> with dE/dx(t_W) = -J x(t_W): the
    reverse sweep is the transpose of the tangent-linear map."""
    N, R, M, W = 35, 4, 300, 40
    J = I.sk_gauss(N, 72).astype(np.float64)
    rng = np.random.default_rng(10)
    x0 = rng.uniform(-0.2, 0.2, size=(R, N))
    u = rng.standard_normal((R, N))
    kw = dict(c=0.3, dt=0.5, M=M, A=0.25)
    E, gx, _, _ = O.relaxed_energy_grad(J, "gbsb", x0, W=W, **kw)
    t = O.tangent_run(J, "gbsb", x0, 0 * x0, u, nsteps=W, renorm_every=10 ** 6, **kw)
    du = t["dx"] * np.exp(t["log_sum"])[:, None]
    lhs = np.sum(gx * u, axis=1)
    rhs = np.sum(-(t["x"] @ J) * du, axis=1)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-10)


# ------------------------------------------------------------- 16-bit JX grid

def test_jx16_grid_scale_and_rounding_by_hand():
    """The paper's JX module works in 16-bit fixed point (Sec. VI, Fig. 2
    caption): x enters the coupling as rint(x 2^15) 2^-15. A coupled pair
    (J = [[0, 1], [1, 0]]) started on grid midpoints x0 = (3, 5) 2^-16 takes
    v = (rint 1.5, rint 2.5) 2^-15 = (2, 2) 2^-15 (half to even), so after one
    bSB step y1 = -(p(t_1) x0 - c v_swap) dt, computed here by hand."""
    J = np.array([[0.0, 1.0], [1.0, 0.0]])
    x0 = np.array([[3.0, 5.0]]) * 2.0 ** -16
    c, dt, M = 0.5, 0.25, 10
    o = O.run(J, "bsb", x0, 0 * x0, c=c, dt=dt, M=M, nsteps=1, jx16=True)
    p1 = 1.0 - 1.0 / M
    v = np.array([2.0, 2.0]) * 2.0 ** -15
    y1 = -(p1 * x0[0] - c * v[::-1]) * dt
    np.testing.assert_array_equal(o["y"][0], y1)
    np.testing.assert_array_equal(o["x"][0], x0[0] + y1 * dt)
    # the exact coupling differs: (x1, x0) instead of the rounded grid values
    e = O.run(J, "bsb", x0, 0 * x0, c=c, dt=dt, M=M, nsteps=1)
    assert not np.array_equal(e["y"], o["y"])


def test_jx16_equals_exact_coupling_on_the_grid_and_bounds_the_error_off_it():
    """x on the 2^-15 grid: the 16-bit coupling is the exact one (first step
    bit-identical). x anywhere: one step's y differs from the exact coupling's
    by at most c dt 2^-16 sum_j |J_ij| (half a grid step per term), and by more
    than a quarter of that somewhere (the grid really is 2^-15)."""
    N, R = 64, 8
    J = I.sk_pm1(N, 3).astype(np.float64)
    c, dt, M = 0.1, 0.5, 100
    xg = np.round(O.init_uniform(R, N, 4) * 2.0 ** 15) * 2.0 ** -15
    a = O.run(J, "gbsb", xg, 0 * xg, c=c, dt=dt, M=M, A=0.2, nsteps=1, jx16=True)
    b = O.run(J, "gbsb", xg, 0 * xg, c=c, dt=dt, M=M, A=0.2, nsteps=1)
    np.testing.assert_array_equal(a["x"], b["x"])
    x0 = O.init_uniform(R, N, 5)
    a = O.run(J, "bsb", x0, 0 * x0, c=c, dt=dt, M=M, nsteps=1, jx16=True)
    b = O.run(J, "bsb", x0, 0 * x0, c=c, dt=dt, M=M, nsteps=1)
    bound = c * dt * 2.0 ** -16 * np.abs(J).sum(axis=1)
    d = np.abs(a["y"] - b["y"])
    assert np.all(d <= bound[None, :] * (1 + 1e-12))
    assert d.max() > 0.25 * bound.max() * 2.0 ** -3  # well above FP64 rounding
    with pytest.raises(ValueError):
        O.run(J, "dsb", x0, 0 * x0, c=c, dt=dt, M=M, nsteps=1, jx16=True)
