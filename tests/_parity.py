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
