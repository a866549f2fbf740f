"""Shared helpers for the GPU-vs-oracle parity tests."""
import numpy as np

# Per test: how many replicas were judged under a widened bar or excused as
# decision near-ties, out of how many compared. Printed in the terminal
# summary of the run (tests/conftest.py).
WIDENED = []


def note_widened(what, n_widened, n_total, how):
    WIDENED.append((str(what), int(n_widened), int(n_total), str(how)))

# FP32 trajectories over the first 50 steps, before chaos decorrelates them:
# max |gpu - oracle| <= RTOL * max |oracle| for each of x, y, p.
RTOL_TRAJ = 1e-5


def assert_traj_close(gpu, ref, rtol=RTOL_TRAJ, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape, (what, gpu.shape, ref.shape)
    scale = max(float(np.max(np.abs(ref))), 1e-30)
    err = float(np.max(np.abs(gpu - ref)))
    assert err <= rtol * scale, f"{what}: max abs err {err:.3e} > {rtol:g} * {scale:.3e}"
    return err / scale


def spins(x):
    return np.where(np.asarray(x) >= 0, 1, -1).astype(np.int8)


def bf16_rne(a):
    """FP32 values rounded to bf16 (8 significant bits) to nearest, ties to even,
    returned as FP32: add just under half an ulp plus the kept part's lowest
    bit to the bit pattern and clear the low 16 bits (finite inputs)."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(np.shape(a))


def bf16_split_sum(J):
    """J_hi + J_lo in FP64 with J_hi = bf16(J) and J_lo = bf16(J - J_hi): the
    matrix whose products the split-bf16 form computes (its sgn-coupled
    products exactly, up to FP32 accumulation)."""
    hi = bf16_rne(J)
    lo = bf16_rne(np.asarray(J, dtype=np.float32) - hi)
    return hi.astype(np.float64) + lo.astype(np.float64)


# A replica whose oracle trajectory put a wall test or a sign within this
# distance of its threshold may legitimately take the other branch in FP32.
TIE_MARGIN = 2e-6


def assert_replicas_close(gpu, ref, margin, rtol=RTOL_TRAJ, rtol_max=None, what="",
                          max_excused=0.25):
    """Per-replica trajectory parity ("relative 1e-5" read norm-wise):
    every replica whose decision margin (from the oracle) is at least
    TIE_MARGIN must satisfy ||gpu - oracle||_2 <= rtol ||oracle||_2, and no
    element may differ by more than rtol_max * max|oracle| (default 10 rtol).
    Replicas with a smaller margin are excused (FP32 may take the other side
    of a wall test or a sign there); at most max_excused of them."""
    if rtol_max is None:
        rtol_max = 10 * rtol
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape
    scale = max(float(np.max(np.abs(ref))), 1e-30)
    diff = gpu - ref
    norm_err = np.linalg.norm(diff, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-30)
    max_err = np.max(np.abs(diff), axis=1)
    checked = np.asarray(margin) >= TIE_MARGIN
    note_widened(what, int((~checked).sum()), len(checked), "excused: near-tie decision")
    assert checked.mean() >= 1.0 - max_excused, (
        f"{what}: {int((~checked).sum())} of {len(checked)} replicas are near-ties")
    if checked.any():
        worst_norm = float(norm_err[checked].max())
        worst_max = float(max_err[checked].max())
        assert worst_norm <= rtol, f"{what}: norm-wise relative error {worst_norm:.3e} > {rtol:g}"
        assert worst_max <= rtol_max * scale, (
            f"{what}: max abs error {worst_max:.3e} > {rtol_max:g} * {scale:.3e}")
        return worst_norm, int((~checked).sum())
    return 0.0, int((~checked).sum())


def assert_one_step_close(state0, gpu1, ref1, J, variant, c, dt, margin, eps=1e-5,
                          what="", max_excused=0.1):
    """One re-synchronised step: every element of y(t_{m+1}), x(t_{m+1}) must
    agree with the oracle to eps relative to the magnitudes of the operands of
    its update (Eq. 3: |y| + dt |p x| + c dt sum_j |J_ij v_j|; Eq. 4 adds |x|),
    the usual forward error model of FP32 arithmetic; p to eps |p|. Replicas
    with a decision near-tie (margin) are excused."""
    x0 = np.asarray(state0["x"], np.float64)
    y0 = np.asarray(state0["y"], np.float64)
    v = np.where(x0 >= 0, 1.0, -1.0) if variant in ("dsb", "gdsb") else x0
    absJ = np.abs(J.dense) if hasattr(J, "dense") and J.dense is not None else None
    if absJ is None and hasattr(J, "rowptr"):
        from scipy.sparse import csr_matrix
        absJ = csr_matrix((np.abs(J.val), J.col, J.rowptr), shape=(J.N, J.N))
    if absJ is None:
        absJ = np.abs(np.asarray(J, np.float64))
    coup = np.asarray(absJ @ np.abs(v).T).T  # sum_j |J_ij v_j|, R x N
    p1 = np.asarray(ref1["p"], np.float64)
    mag_y = np.abs(y0) + dt * np.abs(p1 * x0) + c * dt * coup
    mag_x = np.abs(x0) + dt * mag_y
    checked = np.asarray(margin) >= TIE_MARGIN
    note_widened(what, int((~checked).sum()), len(checked), "excused: near-tie decision")
    assert checked.mean() >= 1.0 - max_excused, f"{what}: too many near-tie replicas"
    # Eq. 7 subtracts (1 - A x^2) p / (M - m) from p: its operands bound the error
    p0 = np.asarray(state0["p"], np.float64)
    mag_p = np.abs(p0) + np.abs(p0 - p1) + np.abs(p1)
    # an element whose wall test (Eq. 5) one side took and the other side missed
    # by less than the bar itself (eps x its operand magnitude) is a tie of the
    # arithmetic's precision, not an error: excused element by element, counted
    xg = np.asarray(gpu1["x"], np.float64)
    yg = np.asarray(gpu1["y"], np.float64)
    xr = np.asarray(ref1["x"], np.float64)
    yr = np.asarray(ref1["y"], np.float64)
    near = lambda v: np.abs(np.abs(v) - 1.0) <= eps * mag_x
    walled = lambda v, w: (np.abs(v) == 1.0) & (w == 0.0)
    tie = (walled(xg, yg) & ~walled(xr, yr) & near(xr)) | (walled(xr, yr) & ~walled(xg, yg) & near(xg))
    if tie.any():
        note_widened(what, int(tie.sum()), tie.size, "elements excused: wall test within the bar")
    for k, mag in (("y", mag_y), ("x", mag_x), ("p", mag_p)):
        err = np.abs(np.asarray(gpu1[k], np.float64) - np.asarray(ref1[k], np.float64))
        bad = (err > eps * mag + 1e-30) & checked[:, None] & ~tie
        assert not bad.any(), (f"{what} {k}: {int(bad.sum())} elements exceed {eps:g} x operand "
                               f"magnitude; worst ratio {float((err / (mag + 1e-30))[checked].max()):.3e}")


def fp32_storage_drift(step_oracle, x0, nsteps):
    """Norm-wise relative drift, per replica, that storing x, y and p in FP32
    between steps causes by itself: the FP64 oracle run straight through versus
    the same oracle restarted every step from its state rounded to FP32.
    step_oracle(x, y, p, m0, nsteps) runs the oracle; returns (reference run,
    drift). Any FP32 implementation of the iteration (the paper's FPGA keeps
    x, y, p in FP32 too) inherits at least this much."""
    ref = step_oracle(x0, 0 * x0, None, 0, nsteps)
    x, y, p = x0, 0 * x0, None
    for m in range(nsteps):
        o = step_oracle(x, y, p, m, 1)
        x, y, p = (o[k].astype(np.float32).astype(np.float64) for k in ("x", "y", "p"))
    d = np.linalg.norm(x - ref["x"], axis=1) / np.maximum(np.linalg.norm(ref["x"], axis=1), 1e-30)
    return ref, d


def assert_within_fp32_drift(gpu_x, ref, drift, base, factor=3.0, margin_min=2e-6):
    """gpu_x (sampled replicas) vs the oracle: norm-wise relative error per
    replica <= max(base, factor * FP32-storage drift); near-tie replicas
    (decision margin below margin_min) are excused."""
    g = np.asarray(gpu_x, np.float64)
    err = np.linalg.norm(g - ref["x"], axis=1) / np.linalg.norm(ref["x"], axis=1)
    tol = np.maximum(base, factor * drift)
    note_widened("fp32-drift bar", int(np.sum(tol > base)), len(tol),
                 f"bar widened to {factor:g} x FP32-storage drift")
    ok = (err <= tol) | (ref["margin"] < margin_min)
    assert ok.all(), f"errors {err[~ok]} vs tolerances {tol[~ok]}"
    return err


def sign_tie_replicas(step_oracle, x0, nsteps, factor=10.0):
    """Which replicas' FP64 trajectories pass a decision (a sign entering the
    coupling, or a wall test) within factor x the deviation that FP32 storage
    of the state has caused by that step: there FP32 arithmetic may take the
    other branch, and a sign flip changes the coupling by 2 c dt |J_ij|, so the
    trajectories part at O(1e-2) for any FP32 implementation. Runs the FP64
    oracle one step at a time beside the same oracle restarted every step from
    its state rounded to FP32 (both oracle-only). step_oracle(x, y, p, m0,
    nsteps) runs the oracle. Returns (FP64 state after nsteps, tie mask)."""
    xa, ya, pa = x0, 0 * x0, None
    xb, yb, pb = x0, 0 * x0, None
    tie = np.zeros(x0.shape[0], bool)
    for m in range(nsteps):
        a = step_oracle(xa, ya, pa, m, 1)
        xa, ya, pa = a["x"], a["y"], a["p"]
        b = step_oracle(xb, yb, pb, m, 1)
        xb, yb, pb = (b[k].astype(np.float32).astype(np.float64) for k in ("x", "y", "p"))
        dev = np.max(np.abs(xa - xb), axis=1)
        tie |= a["margin"] < factor * dev
    return {"x": xa, "y": ya, "p": pa}, tie


def coupling_scale_drift(run_oracle, x0, nsteps, rel=2.0 ** -16):
    """Norm-wise relative drift, per replica, that a systematic relative error
    rel of the coupling causes by itself over nsteps: the FP64 oracle with c
    against the same oracle with c (1 - rel). run_oracle(x0, scale, nsteps)
    runs the oracle with c scaled by `scale`. A split-bf16 coupling has such a
    residue: J_hi + J_lo - J and the dropped J_lo x_lo term are each within
    2^-16 of the products, and the tensor core's FP32 accumulation adds a
    bias of the same order. Oracle-only."""
    ref = run_oracle(x0, 1.0, nsteps)
    pert = run_oracle(x0, 1.0 - rel, nsteps)
    d = np.linalg.norm(pert["x"] - ref["x"], axis=1) / np.maximum(
        np.linalg.norm(ref["x"], axis=1), 1e-30)
    return ref, d
