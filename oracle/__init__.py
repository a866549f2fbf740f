"""Plain FP64 CPU oracle for GbSB / bSB / dSB (arXiv:2508.17655).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may use it; the CUDA library never does. The numeric
work is in ``gsb_oracle.c`` (compiled by ``oracle/build.py``); this module only
marshals numpy arrays through ctypes, plus the paper's closed-form statistics
(TTS, Sec. VI) and the twin-trajectory distance (Eq. 8), which are plain math.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        _LIB = ctypes.CDLL(path)
        _declare(_LIB)
    return _LIB


_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i8p = ctypes.POINTER(ctypes.c_int8)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def _declare(L):
    L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    L.orc_philox4x32_10.restype = None
    L.orc_init_uniform.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                   ctypes.c_uint32, ctypes.c_float, _dp]
    L.orc_init_uniform.restype = None
    L.orc_energy.argtypes = [ctypes.c_int32, _dp, _i32p, _i32p, _dp, _i8p]
    L.orc_energy.restype = ctypes.c_double
    L.orc_energy_batch.argtypes = [ctypes.c_int32, _dp, _i32p, _i32p, _dp, ctypes.c_int32,
                                   _i8p, _dp]
    L.orc_energy_batch.restype = None
    L.orc_cut_dense.argtypes = [ctypes.c_int32, _dp, _i8p]
    L.orc_cut_dense.restype = ctypes.c_double
    L.orc_bruteforce.argtypes = [ctypes.c_int32, _dp, _i8p]
    L.orc_bruteforce.restype = ctypes.c_double
    L.orc_run.argtypes = [ctypes.c_int32, _dp, _i32p, _i32p, _dp, ctypes.c_int32,
                          ctypes.c_int32, _dp, _dp, ctypes.c_double, ctypes.c_double,
                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                          _dp, _dp, _dp, ctypes.c_int32, _dp, _i8p, _i32p, ctypes.c_int32, _dp,
                          _dp]
    L.orc_run.restype = ctypes.c_int
    L.orc_tangent_run.argtypes = [ctypes.c_int32, _dp, _i32p, _i32p, _dp, ctypes.c_int32,
                                  ctypes.c_int32, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                  _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int32, _dp,
                                  ctypes.c_int32]
    L.orc_tangent_run.restype = ctypes.c_int
    L.orc_relaxed_energy_grad.argtypes = [ctypes.c_int32, _dp, ctypes.c_int32, ctypes.c_int32,
                                          _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, _dp, _dp, _dp, _dp,
                                          _dp, ctypes.c_int32, ctypes.c_int32]
    L.orc_relaxed_energy_grad.restype = ctypes.c_int
    L.orc_lambda_extremes.argtypes = [ctypes.c_int32, _dp, _i32p, _i32p, _dp, ctypes.c_int32,
                                      ctypes.c_double, _dp, _dp]
    L.orc_lambda_extremes.restype = None


def _ptr(a, t):
    if a is None:
        return ctypes.cast(None, t)
    return a.ctypes.data_as(t)


class Coupling:
    """J as dense FP64 (N x N, row-major) or as CSR (rowptr, col, val)."""

    def __init__(self, N, dense=None, rowptr=None, col=None, val=None):
        self.N = int(N)
        self.dense = None if dense is None else np.ascontiguousarray(dense, dtype=np.float64)
        self.rowptr = None if rowptr is None else np.ascontiguousarray(rowptr, dtype=np.int32)
        self.col = None if col is None else np.ascontiguousarray(col, dtype=np.int32)
        self.val = None if val is None else np.ascontiguousarray(val, dtype=np.float64)
        if self.dense is None and self.rowptr is None:
            raise ValueError("dense or CSR coupling required")

    def args(self):
        return (ctypes.c_int32(self.N), _ptr(self.dense, _dp), _ptr(self.rowptr, _i32p),
                _ptr(self.col, _i32p), _ptr(self.val, _dp))


def as_coupling(J):
    if isinstance(J, Coupling):
        return J
    J = np.asarray(J, dtype=np.float64)
    return Coupling(J.shape[0], dense=J)


# --------------------------------------------------------------------------
# Philox4x32-10 and the initial-condition draw (App. A)

def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, _u32p), _ptr(k, _u32p), _ptr(out, _u32p))
    return out


def init_uniform(R, N, seed, stream=0, rng=0.1):
    """x_i(0) (stream 0) or y_i(0) (stream 1) uniform in [-rng, rng), R x N."""
    out = np.zeros((R, N), dtype=np.float64)
    lib().orc_init_uniform(R, N, ctypes.c_uint64(seed), stream, ctypes.c_float(rng),
                           _ptr(out, _dp))
    return out


# --------------------------------------------------------------------------
# Energy / cut (Eq. 1; Sec. III)

def energy(J, s):
    C = as_coupling(J)
    s = np.ascontiguousarray(s, dtype=np.int8)
    if s.ndim == 1:
        return lib().orc_energy(*C.args(), _ptr(s, _i8p))
    R = s.shape[0]
    out = np.zeros(R, dtype=np.float64)
    lib().orc_energy_batch(*C.args(), R, _ptr(s, _i8p), _ptr(out, _dp))
    return out


def cut_dense(J, s):
    J = np.ascontiguousarray(J, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.int8)
    return lib().orc_cut_dense(J.shape[0], _ptr(J, _dp), _ptr(s, _i8p))


def total_weight(J):
    """W_tot = sum_{i<j} W_ij with W = -J."""
    C = as_coupling(J)
    if C.dense is not None:
        return -0.5 * float(C.dense.sum())
    return -0.5 * float(C.val.sum())


def bruteforce(J):
    J = np.ascontiguousarray(J, dtype=np.float64)
    N = J.shape[0]
    if N > 30:
        raise ValueError("brute force limited to N <= 30")
    s = np.zeros(N, dtype=np.int8)
    e = lib().orc_bruteforce(N, _ptr(J, _dp), _ptr(s, _i8p))
    return e, s


def lambda_extremes(J, iters=20000, tol=1e-13):
    C = as_coupling(J)
    lmax = ctypes.c_double()
    lmin = ctypes.c_double()
    lib().orc_lambda_extremes(*C.args(), iters, tol, ctypes.byref(lmax), ctypes.byref(lmin))
    return lmax.value, lmin.value


def c_from_lambda(lmax):
    """App. A: c = p(0) / lambda_max = 1 / lambda_max."""
    return 1.0 / lmax


def dt_from_lambda(lmax, lmin, Dt=1.25):
    """Eq. 13: Delta_t = D_t sqrt(2 / (1 - lambda_min / lambda_max))."""
    return Dt * math.sqrt(2.0 / (1.0 - lmin / lmax))


# --------------------------------------------------------------------------
# The iteration (Sec. II, Eqs. 3-7)

VARIANTS = {
    # name: (coupling, control)
    "bsb": (0, 0),
    "gbsb": (0, 1),
    "dsb": (1, 0),
    "gdsb": (1, 1),
}


def run(J, variant, x, y, *, c, dt, M, A=0.0, p=None, sched=None, m0=0, nsteps=None,
        eval_every=0, best=None, nthreads=0, jx16=False):
    """Advance R replicas from step m0 by nsteps (default: to M).

    x, y: R x N arrays (copied). p: R x N (default: ones = p(0), App. A).
    A: scalar or per-replica control strength. jx16: the coupling takes x on the
    16-bit fixed-point grid of the paper's JX module (Sec. VI, Fig. 2 caption).
    Returns a dict with x, y, p, the best-state record (E, s, step) and
    per-replica decision margins (the smallest distance of a wall test, a sign
    or a grid rounding from its threshold; wall_margin: of a wall test alone)."""
    C = as_coupling(J)
    coupling, control = VARIANTS[variant]
    if jx16:
        # the paper's 16-bit fixed-point JX (Sec. VI): x on the 2^-15 grid in the
        # coupling only; the x-coupled variants only
        if coupling != 0:
            raise ValueError("jx16 applies to the x coupling (bSB, GbSB)")
        coupling = 2
    x = np.array(x, dtype=np.float64, copy=True, order="C")
    y = np.array(y, dtype=np.float64, copy=True, order="C")
    R, N = x.shape
    assert N == C.N and y.shape == x.shape
    p = np.ones_like(x) if p is None else np.array(p, dtype=np.float64, copy=True, order="C")
    Aarr = np.broadcast_to(np.asarray(A, dtype=np.float64), (R,)).copy()
    sch = None if sched is None else np.ascontiguousarray(sched, dtype=np.float64)
    if nsteps is None:
        nsteps = M - m0
    if best is None:
        best = {"E": np.full(R, np.inf), "s": np.zeros((R, N), dtype=np.int8),
                "step": np.full(R, -1, dtype=np.int32)}
    else:
        best = {k: np.array(v, copy=True) for k, v in best.items()}
    margin = np.full(R, np.inf)
    wall_margin = np.full(R, np.inf)
    rc = lib().orc_run(*C.args(), coupling, control, _ptr(Aarr, _dp), _ptr(sch, _dp),
                       float(c), float(dt), int(M), int(m0), int(nsteps), int(R),
                       _ptr(x, _dp), _ptr(y, _dp), _ptr(p, _dp), int(eval_every),
                       _ptr(best["E"], _dp), _ptr(best["s"], _i8p),
                       _ptr(best["step"], _i32p), int(nthreads), _ptr(margin, _dp),
                       _ptr(wall_margin, _dp))
    if rc != 0:
        raise ValueError("orc_run rejected its arguments")
    return {"x": x, "y": y, "p": p, "best": best, "margin": margin, "wall_margin": wall_margin}


def tangent_run(J, variant, x, y, dx, *, c, dt, M, A=0.0, p=None, dy=None, dp=None, sched=None,
                m0=0, nsteps=None, renorm_every=10, nthreads=0):
    """Tangent-linear propagation alongside the iteration (FP64). Returns the
    advanced state and tangent and log_sum (per replica, sum of log norms at
    every renormalisation); log_sum / (nsteps dt) is the largest Lyapunov
    exponent estimate."""
    C = as_coupling(J)
    coupling, control = VARIANTS[variant]
    arr = lambda a: np.array(a, dtype=np.float64, copy=True, order="C")
    x, y, dx = arr(x), arr(y), arr(dx)
    R, N = x.shape
    p = np.ones_like(x) if p is None else arr(p)
    dy = np.zeros_like(x) if dy is None else arr(dy)
    dp = np.zeros_like(x) if dp is None else arr(dp)
    Aarr = np.broadcast_to(np.asarray(A, dtype=np.float64), (R,)).copy()
    sch = None if sched is None else np.ascontiguousarray(sched, dtype=np.float64)
    if nsteps is None:
        nsteps = M - m0
    log_sum = np.zeros(R)
    rc = lib().orc_tangent_run(*C.args(), coupling, control, _ptr(Aarr, _dp), _ptr(sch, _dp),
                               float(c), float(dt), int(M), int(m0), int(nsteps), int(R),
                               _ptr(x, _dp), _ptr(y, _dp), _ptr(p, _dp), _ptr(dx, _dp),
                               _ptr(dy, _dp), _ptr(dp, _dp), int(renorm_every),
                               _ptr(log_sum, _dp), int(nthreads))
    if rc != 0:
        raise ValueError("orc_tangent_run rejected its arguments")
    return {"x": x, "y": y, "p": p, "dx": dx, "dy": dy, "dp": dp, "log_sum": log_sum}


def relaxed_energy(J, variant, x0, *, c, dt, M, W, A=0.0):
    """E = -1/2 x(t_W)^T J x(t_W) after W steps from x(0) = x0, y(0) = 0,
    p(0) = 1 (forward only, via orc_run)."""
    J = np.asarray(J, dtype=np.float64)
    x0 = np.asarray(x0, dtype=np.float64)
    o = run(J, variant, x0, 0 * x0, c=c, dt=dt, M=M, A=A, nsteps=W)
    xW = o["x"]
    return -0.5 * np.einsum("ri,ij,rj->r", xW, J, xW), o["margin"]


def relaxed_energy_grad(J, variant, x0, *, c, dt, M, W, A=0.0, nthreads=0, f32_state=False):
    """Reverse-mode gradient of the relaxed energy: (E, dE/dx0, dE/dA, dE/ddt).
    f32_state rounds the stored state to FP32 after every forward step."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    coupling, control = VARIANTS[variant]
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    R, N = x0.shape
    Aarr = np.broadcast_to(np.asarray(A, dtype=np.float64), (R,)).copy()
    E, gA, gdt = np.zeros(R), np.zeros(R), np.zeros(R)
    gx = np.zeros_like(x0)
    rc = lib().orc_relaxed_energy_grad(N, _ptr(J, _dp), coupling, control, _ptr(Aarr, _dp),
                                       float(c), float(dt), int(M), int(W), int(R),
                                       _ptr(x0, _dp), _ptr(E, _dp), _ptr(gx, _dp),
                                       _ptr(gA, _dp), _ptr(gdt, _dp), int(nthreads),
                                       int(bool(f32_state)))
    if rc != 0:
        raise ValueError("orc_relaxed_energy_grad rejected its arguments")
    return E, gx, gA, gdt


def spins(x):
    """s_i = sgn(x_i), with sgn(0) = +1."""
    return np.where(np.asarray(x) >= 0.0, 1, -1).astype(np.int8)


# --------------------------------------------------------------------------
# Statistics (Sec. VI; Table 1 caption)

def success_probability(energies, target, tol=1e-9):
    e = np.asarray(energies, dtype=np.float64)
    return float(np.mean(e <= target + tol))


def ps_error(ps, nrep):
    """Delta P_S = sqrt((P_S - P_S^2) / N_rep)."""
    return math.sqrt(max(ps - ps * ps, 0.0) / nrep)


def tts(ps, t_com, target=0.99):
    """TTS = T_com log(1 - 0.99) / log(1 - P_S), or T_com when P_S > 0.99;
    infinite when P_S == 0."""
    if ps > target:
        return t_com
    if ps <= 0.0:
        return math.inf
    return t_com * math.log(1.0 - target) / math.log(1.0 - ps)


def tts_error(ps, t_com, nrep, target=0.99):
    """Delta_TTS = TTS Delta P_S / [(1 - P_S) |ln(1 - P_S)|] (absolute value as in Sec. VI)."""
    t = tts(ps, t_com, target)
    if not math.isfinite(t) or ps > target:
        return 0.0 if math.isfinite(t) else math.inf
    return t * ps_error(ps, nrep) / ((1.0 - ps) * abs(math.log(1.0 - ps)))


def clopper_pearson(k, n, conf=0.99):
    """Exact binomial confidence interval for k successes in n trials."""
    from scipy.stats import beta
    a = 1.0 - conf
    lo = 0.0 if k == 0 else float(beta.ppf(a / 2, k, n - k + 1))
    hi = 1.0 if k == n else float(beta.ppf(1 - a / 2, k + 1, n - k))
    return lo, hi


def twin_delta(x1, x2):
    """Eq. 8: delta = sqrt(sum_i (x1_i - x2_i)^2 / (4N)), per replica row."""
    d = np.asarray(x1, dtype=np.float64) - np.asarray(x2, dtype=np.float64)
    N = d.shape[-1]
    return np.sqrt(np.sum(d * d, axis=-1) / (4.0 * N))


def twin_initial(R, N, seed):
    """Sec. IV initial conditions: x1 = +-0.1 (random sign), x2 = x1 +- 2e-6
    (random sign), y = 0. Signs come from Philox (streams 2 and 3)."""
    u1 = init_uniform(R, N, seed, stream=2, rng=1.0)
    u2 = init_uniform(R, N, seed, stream=3, rng=1.0)
    x1 = np.where(u1 >= 0.0, 0.1, -0.1)
    x2 = x1 + np.where(u2 >= 0.0, 2e-6, -2e-6)
    return x1, x2


def _load_library_for_tests(path):
    """Swap the loaded oracle library (used only by the mutation test, which
    compiles deliberately broken copies of the oracle to show the pins fail)."""
    global _LIB
    old = _LIB
    L = ctypes.CDLL(path)
    _declare(L)
    _LIB = L
    return old


def _restore_library_for_tests(old):
    global _LIB
    _LIB = old
