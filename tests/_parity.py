"""Shared helpers for the GPU-vs-oracle parity tests."""
import numpy as np

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
