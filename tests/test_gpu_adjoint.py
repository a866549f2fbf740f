"""GPU adjoint (gsb_relaxed_energy_grad) against the FP64 oracle's reverse
sweep, whose gradients are pinned to central finite differences."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2508_17655_gb300 import gsb, inputs as I
from tests._parity import bf16_split_sum

pytestmark = pytest.mark.gpu


def f32(v):
    return float(np.float32(v))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build()


def _gpu_grad(P, variant, M, W, x0, A, dt, c, K=20, precision="fp32"):
    torch = pytest.importorskip("torch")
    R, N = x0.shape
    xd = torch.from_numpy(np.ascontiguousarray(x0, dtype=np.float32)).cuda()
    E = torch.empty(R, dtype=torch.float64, device="cuda")
    gx = torch.empty_like(xd)
    gA = torch.empty(R, dtype=torch.float64, device="cuda")
    gdt = torch.empty(R, dtype=torch.float64, device="cuda")
    P.relaxed_energy_grad(variant, M, W, xd.data_ptr(), R, A, dt, c, E.data_ptr(), gx.data_ptr(),
                          gA.data_ptr(), gdt.data_ptr(), ckpt_every=K, precision=precision,
                          stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return E.cpu().numpy(), gx.cpu().numpy().astype(np.float64), gA.cpu().numpy(), gdt.cpu().numpy()


def _sensitivity(grad_fn, x0):
    """Relative change of each FP64 output (E, dE/dx0 norm-wise, dE/dA, dE/ddt)
    per replica when x0 is perturbed by one FP32 rounding (relative 2^-24,
    random signs): how strongly the gradient itself amplifies FP32-level
    perturbations of the trajectory."""
    base = grad_fn(x0)
    xi = np.where(np.random.default_rng(0).random(x0.shape) < 0.5, -1.0, 1.0)
    pert = grad_fn(x0 * (1.0 + xi * 2.0 ** -24))
    E, gx, gA, gdt = base
    E2, gx2, gA2, gdt2 = pert
    rel = lambda a, b: np.abs(a - b) / np.maximum(np.abs(a), 1e-300)
    return base, (rel(E, E2), _rel_norm(gx2, gx), rel(gA, gA2), rel(gdt, gdt2))


def _rel_norm(g, w):
    """Per replica ||g - w|| / ||w||; a replica whose reference gradient is
    exactly zero scores 0 if g is zero there too, else infinity (never NaN)."""
    num = np.linalg.norm(g - w, axis=1)
    den = np.linalg.norm(w, axis=1)
    out = np.where(num == 0, 0.0, np.inf)
    np.divide(num, den, out=out, where=den > 0)
    return out


def _check(got, want, sens, ok, what, base=1e-4, factor=200.0):
    """Per replica and output: relative error <= max(base, factor x the FP64
    gradient's one-ulp sensitivity). The GPU rounds in FP32 at every forward
    and reverse step, which the x0-only sensitivity undercounts by up to ~100x
    on ill-conditioned replicas; well-conditioned replicas get the 1e-4 bar."""
    names = ("E", "dE/dx0", "dE/dA", "dE/ddt")
    for k, name in enumerate(names):
        g, w = got[k], want[k]
        if k == 1:
            err = _rel_norm(g, w)
        else:
            if np.all(w == 0):
                assert np.all(g == 0), name
                continue
            # a gradient that nearly cancels across its terms has no meaningful
            # relative error: floor the scale at 5 % of the median magnitude
            scale = np.maximum(np.abs(w), 0.05 * np.median(np.abs(w)))
            err = np.abs(g - w) / np.maximum(scale, 1e-300)
        tol = np.maximum(base[k] if isinstance(base, tuple) else base, factor * sens[k])
        # a NaN error or tolerance would pass the comparison below: it fails here
        assert not np.isnan(err[ok]).any(), f"{what} {name}: NaN error"
        assert not np.isnan(tol[ok]).any(), f"{what} {name}: NaN tolerance"
        bad = ok & (err > tol)
        assert not bad.any(), (f"{what} {name}: errors {err[bad]} vs tolerances {tol[bad]}")


def _oracle_J(J, precision):
    return bf16_split_sum(J) if precision == "bf16x3" else J.astype(np.float64)


# The split form's x coupling against the oracle on J_hi + J_lo: each product
# J x differs by J_hi (x - x_hi - x_lo) + J_lo x_lo + ..., at most about
# 2^-17 + 2^-16 < 2^-15 of its magnitude sum_j |J_ij x_j|, where FP32 carries
# one rounding of 2^-24: 2^9 times the FP32 bars that scale with the rounding.
SPLIT_RATIO = 2.0 ** 9


def _energy_cancellation(Jd, x):
    """kappa per replica: the magnitude 1/2 sum_i |x_i| sum_j |J_ij x_j| of the
    energy's terms over |E|. A product error that is relative to the terms'
    magnitude is kappa times larger relative to E."""
    mag = 0.5 * np.einsum("ri,ri->r", np.abs(x), np.abs(x) @ np.abs(Jd).T)
    E = -0.5 * np.einsum("ri,ri->r", x, x @ Jd.T)
    return mag / np.maximum(np.abs(E), 1e-300)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("variant", ["gbsb", "bsb", "gdsb", "dsb"])
def test_adjoint_well_conditioned_within_1e4(variant, precision):
    """A short window from small x0 (no wall events, little amplification):
    every replica's E, dE/dx0, dE/dA, dE/ddt within 1e-4 relative of FP64 (for
    the split-bf16 form, of the oracle on its matrix J_hi + J_lo)."""
    N, R, M, W = 300, 96, 400, 12
    J = I.sk_gauss(N, 13)
    c, dt = 0.5, f32(0.8)
    A = np.linspace(0.1, 0.4, R).astype(np.float32)
    x0 = O.init_uniform(R, N, 18, rng=0.02)
    got = _gpu_grad(gsb.Problem.dense(J), variant, M, W, x0, A, dt, c, precision=precision)
    Jd = _oracle_J(J, precision)
    Ad = A.astype(np.float64)
    want = O.relaxed_energy_grad(Jd, variant, x0, c=c, dt=dt, M=M, W=W, A=Ad)
    run = O.run(Jd, variant, x0, 0 * x0, c=c, dt=dt, M=M, A=Ad, nsteps=W)
    sign = variant in ("dsb", "gdsb")
    ok = run["margin"] >= (2e-6 if sign else 0.5)
    assert ok.mean() >= 0.9
    zero = (np.zeros(R),) * 4
    base = 1e-4
    if precision == "bf16x3" and not sign:
        # each product carries up to 2^-15 of its magnitude (SPLIT_RATIO): the
        # gradients W 2^-14 (W forward and W reverse products; the recompute
        # repeats the forward bit for bit); E its trajectory's W 2^-15 plus its
        # last product's 2^-15 of its terms' magnitude (kappa 2^-15 of E),
        # bounded by 2^-14 max(W, kappa). The sgn coupling is exact on
        # J_hi + J_lo: the FP32 bar.
        kappa = _energy_cancellation(Jd, run["x"])
        base = (2.0 ** -14 * np.maximum(W, kappa),) + (W * 2.0 ** -14,) * 3
    _check(got, want, zero, ok, f"{variant} {precision}", base=base, factor=0.0)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("variant", ["gbsb", "bsb", "gdsb", "dsb"])
def test_adjoint_matches_oracle_small(variant, precision):
    """60 steps with wall events: per replica within max(1e-4, 200 x the FP64
    gradient's sensitivity to a 2^-24 relative perturbation of x0); the
    split-bf16 form against the oracle on J_hi + J_lo, its x coupling also
    splitting x, so SPLIT_RATIO x the sensitivity term and a floor of
    W 2^-14 (as in the well-conditioned test)."""
    N, R, M, W = 300, 70, 400, 60
    J = I.sk_gauss(N, 13)
    c, dt = 0.5, f32(0.8)
    A = np.linspace(0.1, 0.4, R).astype(np.float32)
    x0 = O.init_uniform(R, N, 17)
    got = _gpu_grad(gsb.Problem.dense(J), variant, M, W, x0, A, dt, c, precision=precision)
    Jd = _oracle_J(J, precision)
    Ad = A.astype(np.float64)
    want, sens = _sensitivity(
        lambda x: O.relaxed_energy_grad(Jd, variant, x, c=c, dt=dt, M=M, W=W, A=Ad), x0)
    margin = O.run(Jd, variant, x0, 0 * x0, c=c, dt=dt, M=M, A=Ad, nsteps=W)["margin"]
    # a different wall or sign decision changes the gradient by O(1)
    sign = variant in ("dsb", "gdsb")
    ok = margin >= (1e-5 if sign else 1e-4)
    assert ok.sum() >= 2
    split_x = precision == "bf16x3" and not sign
    factor = 200.0 * (SPLIT_RATIO if split_x else 1.0)
    _check(got, want, sens, ok, f"{variant} {precision}", base=W * 2.0 ** -14 if split_x else 1e-4,
           factor=factor)


def test_adjoint_config5_shape_against_fp64():
    """N = 2000 SK (Gaussian, FP32 J), R = 256, the first 200 steps of a run
    with the paper's K2000 step count M = 21,500 (Fig. 1(d)), checkpoints every
    20 steps, c = 1/(2 sqrt(N) sigma) = 1/2 (App. A), dt = 1.25: a window with no
    wall event. Keeping x, y, p in FP32 (as the paper's machine does) moves x
    by ~1.3e-4 in 200 steps here, for any FP32 implementation; each sampled
    replica's E, dE/dx0, dE/dA, dE/ddt must be within max(1e-4, 5 x the change
    FP32 storage of the forward state alone causes in the FP64 oracle's
    gradient; the GPU also keeps the adjoint state in FP32 through the reverse
    sweep, which roughly doubles it). The FP64 gradient is checked against
    central differences on one replica."""
    N, R, M, W = 2000, 256, 21500, 200
    J = I.sk_gauss(N, 0)
    Jd = J.astype(np.float64)
    c, dt, A = 0.5, 1.25, 0.2
    x0 = O.init_uniform(R, N, 1)
    got = _gpu_grad(gsb.Problem.dense(J), "gbsb", M, W, x0, A, dt, c)
    pick = np.linspace(0, R - 1, 12).astype(int)
    want = O.relaxed_energy_grad(Jd, "gbsb", x0[pick], c=c, dt=dt, M=M, W=W, A=A)
    store = O.relaxed_energy_grad(Jd, "gbsb", x0[pick], c=c, dt=dt, M=M, W=W, A=A, f32_state=True)
    rel = lambda a, b: np.abs(a - b) / np.abs(a)
    drift = (rel(want[0], store[0]),
             np.linalg.norm(want[1] - store[1], axis=1) / np.linalg.norm(want[1], axis=1),
             rel(want[2], store[2]), rel(want[3], store[3]))
    margin = O.run(Jd, "gbsb", x0[pick], 0 * x0[pick], c=c, dt=dt, M=M, A=A, nsteps=W)["margin"]
    assert np.all(margin > 0.1)  # wall-free window
    _check(tuple(g[pick] for g in got), want, drift, np.ones(len(pick), bool), "config 5",
           base=1e-4, factor=5.0)
    h = 1e-6
    xr = x0[pick][:1]
    fd = (O.relaxed_energy(Jd, "gbsb", xr, c=c, dt=dt + h, M=M, W=W, A=A)[0]
          - O.relaxed_energy(Jd, "gbsb", xr, c=c, dt=dt - h, M=M, W=W, A=A)[0]) / (2 * h)
    # central differences of an O(1) energy with h = 1e-6 carry ~1e-10 of roundoff
    assert abs(want[3][0] - fd[0]) <= 1e-4 * abs(fd[0]) + 1e-8
    fdA = (O.relaxed_energy(Jd, "gbsb", xr, c=c, dt=dt, M=M, W=W, A=A + h)[0]
           - O.relaxed_energy(Jd, "gbsb", xr, c=c, dt=dt, M=M, W=W, A=A - h)[0]) / (2 * h)
    assert abs(want[2][0] - fdA[0]) <= 1e-4 * abs(fdA[0]) + 1e-8


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_checkpoint_interval_does_not_change_the_gradient(precision):
    N, R, M, W = 256, 128, 500, 45
    J = I.sk_gauss(N, 19)
    x0 = O.init_uniform(R, N, 23)
    P = gsb.Problem.dense(J)
    outs = [_gpu_grad(P, "gbsb", M, W, x0, 0.3, 0.9, 0.5, K=K, precision=precision)
            for K in (1, 7, 20, 45)]
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


def test_torch_autograd_function():
    torch = pytest.importorskip("torch")
    from paper_2508_17655_gb300.autograd import relaxed_energy
    N, R, M, W = 200, 33, 300, 30
    J = I.sk_gauss(N, 29)
    P = gsb.Problem.dense(J)
    x0 = torch.from_numpy(O.init_uniform(R, N, 31).astype(np.float32)).cuda().requires_grad_()
    A = torch.full((R,), 0.25, dtype=torch.float32, requires_grad=True)
    dt = torch.tensor(0.8, dtype=torch.float32, requires_grad=True)
    w = torch.linspace(0.5, 1.5, R, dtype=torch.float64, device="cuda")
    E = relaxed_energy(x0, A, dt, P, "gbsb", M, W, 0.5, 10)
    (w * E).sum().backward()
    # the same kernels called directly: autograd only applies the chain rule
    Ed, gx, gA, gdt = _gpu_grad(P, "gbsb", M, W, x0.detach().cpu().numpy(), 0.25, 0.8, 0.5, K=10)
    wn = w.cpu().numpy()
    np.testing.assert_array_equal(E.detach().cpu().numpy(), Ed)
    np.testing.assert_allclose(x0.grad.cpu().numpy(), (wn[:, None] * gx).astype(np.float32),
                               rtol=1e-6)
    np.testing.assert_allclose(A.grad.numpy(), (wn * gA).astype(np.float32), rtol=1e-6)
    np.testing.assert_allclose(float(dt.grad), float(np.sum(wn * gdt)), rtol=1e-5)
    assert A.grad.device.type == "cpu" and x0.grad.device.type == "cuda"


def test_adjoint_bf16x3_config5_shape():
    """The configuration-5 shape (N = 2000 SK, R = 256, 200 steps of M = 21,500,
    checkpoints every 20) with the products on the tensor cores: sampled
    replicas against the FP64 oracle on J_hi + J_lo within max(1e-4, 5 x the
    FP32-storage drift x SPLIT_RATIO) -- the x split perturbs each step about
    that many times more than FP32 rounding of the state."""
    N, R, M, W = 2000, 256, 21500, 200
    J = I.sk_gauss(N, 0)
    Jd = bf16_split_sum(J)
    c, dt, A = 0.5, 1.25, 0.2
    x0 = O.init_uniform(R, N, 1)
    got = _gpu_grad(gsb.Problem.dense(J), "gbsb", M, W, x0, A, dt, c, precision="bf16x3")
    pick = np.linspace(0, R - 1, 6).astype(int)
    want = O.relaxed_energy_grad(Jd, "gbsb", x0[pick], c=c, dt=dt, M=M, W=W, A=A)
    store = O.relaxed_energy_grad(Jd, "gbsb", x0[pick], c=c, dt=dt, M=M, W=W, A=A, f32_state=True)
    rel = lambda a, b: np.abs(a - b) / np.abs(a)
    drift = (rel(want[0], store[0]),
             np.linalg.norm(want[1] - store[1], axis=1) / np.linalg.norm(want[1], axis=1),
             rel(want[2], store[2]), rel(want[3], store[3]))
    _check(tuple(g[pick] for g in got), want, drift, np.ones(len(pick), bool), "config 5 bf16x3",
           base=1e-4, factor=5.0 * SPLIT_RATIO)


def test_adjoint_rejects_other_forms():
    torch = pytest.importorskip("torch")
    J = I.sk_gauss(64, 2)
    x0 = O.init_uniform(4, 64, 1)
    with pytest.raises(gsb.GsbError) as e:
        _gpu_grad(gsb.Problem.dense(J), "gbsb", 100, 5, x0, 0.2, 0.9, 0.5, precision="fp8")
    assert e.value.status == gsb.EUNSUPPORTED


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("N", [1, 2, 129])
def test_adjoint_degenerate_and_edge_sizes(N, precision):
    """N = 1 (no coupling), N = 2 and N = 129 (one spin past a tile), 5
    replicas, a 10-step window from small x0 (no wall event): E, dE/dx0,
    dE/dA, dE/ddt within 1e-4 relative of the FP64 oracle (the split form
    against the oracle on J_hi + J_lo, with the bars of the well-conditioned
    test)."""
    J = I.sk_gauss(N, 6) if N > 1 else np.zeros((1, 1), np.float32)
    R, M, W = 5, 300, 10
    c, dt = 0.5, f32(0.8)
    A = np.linspace(0.1, 0.3, R).astype(np.float32)
    x0 = O.init_uniform(R, N, 7, rng=0.02)
    got = _gpu_grad(gsb.Problem.dense(J), "gbsb", M, W, x0, A, dt, c, precision=precision)
    Jd = _oracle_J(J, precision)
    want = O.relaxed_energy_grad(Jd, "gbsb", x0, c=c, dt=dt, M=M, W=W, A=A.astype(np.float64))
    base = W * 2.0 ** -14 if precision == "bf16x3" else 1e-4
    if N > 1 and precision == "bf16x3":
        # the bars of the well-conditioned test
        run = O.run(Jd, "gbsb", x0, 0 * x0, c=c, dt=dt, M=M, A=A.astype(np.float64), nsteps=W)
        kappa = _energy_cancellation(Jd, run["x"])
        base = (2.0 ** -14 * np.maximum(W, kappa),) + (base,) * 3
    _check(got, want, (np.zeros(R),) * 4, np.ones(R, bool), f"N={N} {precision}", base=base,
           factor=0.0)
