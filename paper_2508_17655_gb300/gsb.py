"""Thin ctypes binding of libgsb (include/gsb.h). Argument marshalling only:
every step of the method runs in the library's CUDA kernels.

The library must exist (``paper_2508_17655_gb300.build.build()``); importing
this module without it raises, there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

# enums / flags of include/gsb.h
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, ENUMERIC, ENODEV = range(8)
BSB, GBSB, DSB, GDSB = range(4)
PREC_AUTO, PREC_FP32, PREC_FP8, PREC_FX32, PREC_BF16X3, PREC_FX16 = range(6)
J_DENSE_I8, J_DENSE_F32, J_CSR_F32 = range(3)
CREATE_DEVICE_INPUT, CREATE_NO_VALIDATE = 0x1, 0x2
RUN_DEFER, RUN_PROFILE, RUN_SM_PAIRS, RUN_FUSED_CSR = 0x1, 0x2, 0x4, 0x8

VARIANT = {"bsb": BSB, "gbsb": GBSB, "dsb": DSB, "gdsb": GDSB}
PRECISION = {"auto": PREC_AUTO, "fp32": PREC_FP32, "fp8": PREC_FP8, "fx32": PREC_FX32,
             "bf16x3": PREC_BF16X3, "fx16": PREC_FX16}


class gsb_params(ctypes.Structure):
    _fields_ = [
        ("variant", ctypes.c_int32),
        ("M", ctypes.c_int32),
        ("R", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("c", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("A", ctypes.c_float),
        ("A_per_replica", ctypes.POINTER(ctypes.c_float)),
        ("schedule", ctypes.POINTER(ctypes.c_float)),
        ("seed", ctypes.c_uint64),
        ("x0_range", ctypes.c_float),
        ("y0_uniform", ctypes.c_int32),
        ("eval_every", ctypes.c_int32),
        ("steps_per_launch", ctypes.c_int32),
        ("x0", ctypes.POINTER(ctypes.c_float)),
        ("y0", ctypes.POINTER(ctypes.c_float)),
        ("flags", ctypes.c_uint32),
    ]


class gsb_batch_info(ctypes.Structure):
    _fields_ = [
        ("force_tile", ctypes.c_int32),
        ("max_steps", ctypes.c_int32),
        ("tile", ctypes.c_int32),
        ("steps_per_graph", ctypes.c_int32),
        ("tiles", ctypes.c_int32),
        ("ms_step_tile128", ctypes.c_double),
        ("ms_step_tile64", ctypes.c_double),
        ("force_tiles_per_cta", ctypes.c_int32),
        ("tiles_per_cta", ctypes.c_int32),
        ("windows", ctypes.c_int32),
        ("ctas", ctypes.c_int32),
        ("ms_step_probe", ctypes.c_double * 4),
        ("graphed", ctypes.c_int32),
    ]


class GsbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libgsb status {status}: {msg}")
        self.status = status


_LIB = None
_vp = ctypes.c_void_p


def library_path():
    """The library this process loads: the release build, or the debug build
    (device-side bounds checks, -DGSB_DEBUG) when GSB_LIBRARY=debug."""
    return _build.LIB_DEBUG if os.environ.get("GSB_LIBRARY") == "debug" else _build.LIB


def lib():
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libgsb.so is not built ({path}); run "
                               "paper_2508_17655_gb300.build.build() first")
        L = ctypes.CDLL(path)
        _declare(L)
        _LIB = L
    return _LIB


def _declare(L):
    st = ctypes.c_int
    fp = ctypes.POINTER(ctypes.c_float)
    L.gsb_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.c_int32, _vp,
                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), fp,
                             ctypes.c_int64, fp, ctypes.c_uint32, _vp]
    L.gsb_create.restype = st
    L.gsb_qubo_to_ising.argtypes = [ctypes.c_int32, fp, fp, fp, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)]
    L.gsb_qubo_to_ising.restype = st
    L.gsb_create_qubo.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, _vp, ctypes.c_uint32,
                                  ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), _vp]
    L.gsb_create_qubo.restype = st
    L.gsb_destroy.argtypes = [_vp]
    L.gsb_destroy.restype = st
    L.gsb_problem_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double), _vp]
    L.gsb_problem_info.restype = st
    L.gsb_run.argtypes = [_vp, ctypes.POINTER(gsb_params), ctypes.POINTER(_vp), _vp]
    L.gsb_run.restype = st
    L.gsb_run_steps.argtypes = [_vp, ctypes.c_int32]
    L.gsb_run_steps.restype = st
    L.gsb_best.argtypes = [_vp, ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]
    L.gsb_best.restype = st
    L.gsb_get_state.argtypes = [_vp, fp, fp, fp, ctypes.POINTER(ctypes.c_int32)]
    L.gsb_get_state.restype = st
    L.gsb_energy.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int8),
                             ctypes.POINTER(ctypes.c_double), _vp]
    L.gsb_energy.restype = st
    L.gsb_run_restart.argtypes = [_vp, ctypes.c_uint64, ctypes.c_uint32]
    L.gsb_run_restart.restype = st
    L.gsb_kernel_time.argtypes = [_vp, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.gsb_kernel_time.restype = st
    L.gsb_run_kernel.argtypes = [_vp]
    L.gsb_run_kernel.restype = ctypes.c_char_p
    L.gsb_lyapunov.argtypes = [_vp, ctypes.POINTER(gsb_params), ctypes.c_int32,
                               ctypes.POINTER(ctypes.c_float), ctypes.c_int32, ctypes.c_int32,
                               ctypes.POINTER(ctypes.c_double), _vp]
    L.gsb_lyapunov.restype = st
    L.gsb_twin_run.argtypes = [_vp, ctypes.POINTER(gsb_params), ctypes.c_int32,
                               ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_vp), _vp]
    L.gsb_twin_run.restype = st
    L.gsb_twin_delta.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
    L.gsb_twin_delta.restype = st
    L.gsb_relaxed_energy_grad.argtypes = [_vp, ctypes.POINTER(gsb_params), ctypes.c_int32,
                                          ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp]
    L.gsb_relaxed_energy_grad.restype = st
    L.gsb_batch_run.argtypes = [ctypes.c_int32, ctypes.POINTER(_vp), ctypes.POINTER(gsb_params),
                                ctypes.POINTER(_vp), ctypes.POINTER(gsb_batch_info), _vp]
    L.gsb_batch_run.restype = st
    L.gsb_energy_noalloc.argtypes = [_vp, ctypes.c_int32, _vp, ctypes.c_int32, _vp, _vp]
    L.gsb_energy_noalloc.restype = st
    L.gsb_run_destroy.argtypes = [_vp]
    L.gsb_run_destroy.restype = st
    L.gsb_run_set_state.argtypes = [_vp, ctypes.POINTER(ctypes.c_float),
                                    ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                    ctypes.c_int32, ctypes.POINTER(ctypes.c_int8),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]
    L.gsb_run_set_state.restype = st
    L.gsb_set_memory_limit.argtypes = [ctypes.c_int64]
    L.gsb_set_memory_limit.restype = st
    L.gsb_memory_usage.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.gsb_memory_usage.restype = st
    L.gsb_release_cached_memory.argtypes = []
    L.gsb_release_cached_memory.restype = st
    L.gsb_wait_check.argtypes = [ctypes.c_int32, ctypes.c_int64, _vp]
    L.gsb_wait_check.restype = st
    L.gsb_debug_build.argtypes = []
    L.gsb_debug_build.restype = ctypes.c_int32
    L.gsb_debug_selftest.argtypes = []
    L.gsb_debug_selftest.restype = st
    L.gsb_set_call_profiling.argtypes = [ctypes.c_int32]
    L.gsb_set_call_profiling.restype = st
    L.gsb_last_call_profile.argtypes = [ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64)]
    L.gsb_last_call_profile.restype = st
    L.gsb_last_error.argtypes = []
    L.gsb_last_error.restype = ctypes.c_char_p
    L.gsb_version.restype = ctypes.c_int32
    L.gsb_launch_count.restype = ctypes.c_int64


def _check(status):
    if status != OK:
        raise GsbError(status, lib().gsb_last_error().decode())


def _p(a, ctype):
    if a is None:
        return ctypes.cast(None, ctypes.POINTER(ctype))
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def release_cached_memory():
    """Return the device blocks the library keeps for reuse to CUDA."""
    _check(lib().gsb_release_cached_memory())


def set_memory_limit(nbytes):
    """Cap on the device bytes the library's problems and runs hold (0: none)."""
    _check(lib().gsb_set_memory_limit(int(nbytes)))


def memory_usage():
    """(bytes held by live problems and runs, bytes kept for reuse)."""
    a = ctypes.c_int64()
    b = ctypes.c_int64()
    _check(lib().gsb_memory_usage(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def wait_check(kind, limit_ns, stream=None):
    """gsb_wait_check: one bounded device-side wait (0: mbarrier, 1: counter,
    both never satisfied; 2: a counter already at its target). Raises GsbError
    with status ETIMEOUT when the wait gives up."""
    _check(lib().gsb_wait_check(int(kind), int(limit_ns), _stream_handle(stream)))


def debug_build():
    """gsb_debug_build: True when this process loaded the -DGSB_DEBUG library
    (device-side bounds checks; GSB_LIBRARY=debug)."""
    return bool(lib().gsb_debug_build())


def debug_selftest():
    """gsb_debug_selftest (debug build): kernels run on inputs planted to fail
    their bounds checks; raises GsbError unless both checks fired."""
    _check(lib().gsb_debug_selftest())


def set_call_profiling(on):
    """gsb_set_call_profiling: CUDA events around the step-kernel launches of
    this thread's later batch / Lyapunov / gradient calls."""
    _check(lib().gsb_set_call_profiling(int(bool(on))))


def last_call_profile():
    """(device ms of the step-kernel launches, launches, time steps covered) of
    this thread's last profiled batch / Lyapunov / gradient call."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    k = ctypes.c_int64()
    _check(lib().gsb_last_call_profile(ctypes.byref(ms), ctypes.byref(n), ctypes.byref(k)))
    return ms.value, n.value, k.value


def launch_count():
    return int(lib().gsb_launch_count())


def _make_params(variant, M, R, *, c=0.0, dt=0.0, A=0.0, seed=0, precision="auto",
                 eval_every=0, y0_uniform=False, x0_range=0.0):
    prm = gsb_params()
    prm.variant = VARIANT[variant] if isinstance(variant, str) else int(variant)
    prm.M = int(M)
    prm.R = int(R)
    prm.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    prm.c = float(c)
    prm.dt = float(dt)
    prm.A = float(A)
    prm.seed = int(seed)
    prm.eval_every = int(eval_every)
    prm.y0_uniform = int(bool(y0_uniform))
    prm.x0_range = float(x0_range)
    return prm


class _BatchRun(object):
    """A run handle produced by gsb_batch_run (same queries as Run)."""

    def __init__(self, problem, handle, R):
        self.problem = problem
        self.handle = handle
        self.R = int(R)
        self.N = problem.N

    best = None  # filled below from Run
    state = None
    _n_state = None
    close = None
    __del__ = None


def batch_run(problems, specs, force_tile=0, max_steps=0, force_tiles_per_cta=0, stream=None):
    """Run len(problems) instances together (gsb_batch_run). specs: list of
    dicts with the keyword arguments of Problem.run (variant, M, R, c, dt, A,
    seed, precision, ...). Returns (runs, info dict)."""
    n = len(problems)
    prms = (gsb_params * n)(*[_make_params(**sp) for sp in specs])
    handles = (_vp * n)(*[p.handle for p in problems])
    outs = (_vp * n)()
    info = gsb_batch_info()
    info.force_tile = int(force_tile)
    info.max_steps = int(max_steps)
    info.force_tiles_per_cta = int(force_tiles_per_cta)
    _check(lib().gsb_batch_run(n, handles, prms, outs, ctypes.byref(info),
                               _stream_handle(stream)))
    runs = [_BatchRun(problems[k], _vp(outs[k]), specs[k]["R"]) for k in range(n)]
    return runs, {"tile": info.tile, "steps_per_graph": info.steps_per_graph,
                  "tiles": info.tiles, "ms_step_tile128": info.ms_step_tile128,
                  "ms_step_tile64": info.ms_step_tile64, "tiles_per_cta": info.tiles_per_cta,
                  "windows": info.windows, "ctas": info.ctas,
                  "ms_step_probe": list(info.ms_step_probe), "graphed": info.graphed}


def qubo_to_ising(Q):
    """gsb_qubo_to_ising (host only, no GPU): the Ising form of the QUBO
    f(b) = b^T Q b under s = 2b - 1. Returns (J, h, scale, offset) with
    f(b) = scale * E(s) + offset."""
    Qc = np.ascontiguousarray(Q, dtype=np.float32)
    N = Qc.shape[0]
    J = np.zeros((N, N), dtype=np.float32)
    h = np.zeros(N, dtype=np.float32)
    sc = ctypes.c_double()
    off = ctypes.c_double()
    _check(lib().gsb_qubo_to_ising(N, _p(Qc, ctypes.c_float), _p(J, ctypes.c_float),
                                   _p(h, ctypes.c_float), ctypes.byref(sc), ctypes.byref(off)))
    return J, h, sc.value, off.value


def energy_noalloc(J_ptr, N, spins_ptr, R, energies_ptr, stream=None):
    """gsb_energy_noalloc on caller device buffers (raw pointers, e.g. from
    torch tensors' data_ptr()): J N x N float32, spins R x N int8, energies R
    float64. Allocates nothing on the device."""
    _check(lib().gsb_energy_noalloc(J_ptr, int(N), spins_ptr, int(R), energies_ptr,
                                    _stream_handle(stream)))


class Problem:
    """Device-resident coupling matrix (Eq. 1), dense or CSR."""

    def __init__(self, handle, N):
        self.handle = handle
        self.N = N

    @classmethod
    def dense(cls, J, h=None, stream=None, validate=True):
        J = np.asarray(J)
        N = J.shape[0]
        if J.dtype == np.int8:
            fmt, Jc = J_DENSE_I8, np.ascontiguousarray(J)
        else:
            fmt, Jc = J_DENSE_F32, np.ascontiguousarray(J, dtype=np.float32)
        hc = None if h is None else np.ascontiguousarray(h, dtype=np.float32)
        out = _vp()
        _check(lib().gsb_create(ctypes.byref(out), N, fmt, Jc.ctypes.data_as(_vp), None, None,
                                None, 0, _p(hc, ctypes.c_float),
                                0 if validate else CREATE_NO_VALIDATE, _stream_handle(stream)))
        return cls(out, N)

    @classmethod
    def qubo(cls, Q, stream=None):
        """gsb_create_qubo: the QUBO f(b) = b^T Q b as an Ising problem (with one
        auxiliary spin). Returns the problem; its .scale and .offset give
        f(b) = scale * E + offset for the energies E that runs report, and
        b = (1 + s) / 2 for their spins."""
        Qc = np.ascontiguousarray(Q, dtype=np.float32)
        N = Qc.shape[0]
        out = _vp()
        sc = ctypes.c_double()
        off = ctypes.c_double()
        _check(lib().gsb_create_qubo(ctypes.byref(out), N, Qc.ctypes.data_as(_vp), 0,
                                     ctypes.byref(sc), ctypes.byref(off),
                                     _stream_handle(stream)))
        P = cls(out, N)
        P.scale, P.offset = sc.value, off.value
        return P

    @classmethod
    def csr(cls, N, rowptr, col, val, h=None, stream=None, validate=True):
        rp = np.ascontiguousarray(rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(col, dtype=np.int32)
        vv = np.ascontiguousarray(val, dtype=np.float32)
        hc = None if h is None else np.ascontiguousarray(h, dtype=np.float32)
        out = _vp()
        _check(lib().gsb_create(ctypes.byref(out), N, J_CSR_F32, None, _p(rp, ctypes.c_int32),
                                _p(ci, ctypes.c_int32), _p(vv, ctypes.c_float), len(ci),
                                _p(hc, ctypes.c_float), 0 if validate else CREATE_NO_VALIDATE,
                                _stream_handle(stream)))
        return cls(out, N)

    def info(self, stream=None):
        n = ctypes.c_int32()
        lmax = ctypes.c_double()
        lmin = ctypes.c_double()
        _check(lib().gsb_problem_info(self.handle, ctypes.byref(n), ctypes.byref(lmax),
                                      ctypes.byref(lmin), _stream_handle(stream)))
        return n.value, lmax.value, lmin.value

    def energy(self, spins, stream=None):
        s = np.ascontiguousarray(spins, dtype=np.int8)
        if s.ndim == 1:
            s = s[None]
        out = np.zeros(s.shape[0], dtype=np.float64)
        _check(lib().gsb_energy(self.handle, s.shape[0], _p(s, ctypes.c_int8),
                                _p(out, ctypes.c_double), _stream_handle(stream)))
        return out

    def run(self, variant, M, R, *, c=0.0, dt=0.0, A=0.0, seed=0, precision="auto",
            eval_every=0, x0=None, y0=None, y0_uniform=False, x0_range=0.0, schedule=None,
            steps_per_launch=0, defer=False, profile=False, stream=None, sm_pairs=False,
            fused_csr=False):
        return Run(self, variant, M, R, c=c, dt=dt, A=A, seed=seed, precision=precision,
                   eval_every=eval_every, x0=x0, y0=y0, y0_uniform=y0_uniform,
                   x0_range=x0_range, schedule=schedule, steps_per_launch=steps_per_launch,
                   defer=defer, profile=profile, stream=stream, sm_pairs=sm_pairs,
                   fused_csr=fused_csr)

    def lyapunov(self, variant, M, R, A_values, *, c=0.0, dt=0.0, seed=0, renorm_every=10,
                 nsteps=0, y0_uniform=False, x0_range=0.0, precision="fp32", stream=None):
        """Largest Lyapunov exponent per replica (len(A_values) x R), from the
        tangent-linear kernel; precision "fp32" (CUDA cores) or "bf16x3" (J x
        and J dx on the tensor cores, split bf16); see gsb_lyapunov in
        include/gsb.h."""
        prm = gsb_params()
        prm.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        prm.variant = VARIANT[variant] if isinstance(variant, str) else int(variant)
        prm.M = int(M)
        prm.R = int(R)
        prm.c = float(c)
        prm.dt = float(dt)
        prm.seed = int(seed)
        prm.x0_range = float(x0_range)
        prm.y0_uniform = int(bool(y0_uniform))
        A = np.ascontiguousarray(A_values, dtype=np.float32)
        out = np.zeros(len(A) * int(R), dtype=np.float64)
        _check(lib().gsb_lyapunov(self.handle, ctypes.byref(prm), len(A), _p(A, ctypes.c_float),
                                  int(renorm_every), int(nsteps), _p(out, ctypes.c_double),
                                  _stream_handle(stream)))
        return out.reshape(len(A), int(R))

    def twin_run(self, variant, M, R, A_values, *, c=0.0, dt=0.0, seed=0, precision="auto",
                 eval_every=0, schedule=None, steps_per_launch=0, defer=True, profile=False,
                 stream=None):
        """Twin trajectories of Sec. IV (gsb_twin_run): len(A_values) x R pairs,
        deferred by default; advance with .steps(n), read Eq. 8 with .delta()."""
        return TwinRun(self, variant, M, R, A_values, c=c, dt=dt, seed=seed,
                       precision=precision, eval_every=eval_every, schedule=schedule,
                       steps_per_launch=steps_per_launch, defer=defer, profile=profile,
                       stream=stream)

    def twin_delta(self, variant, M, R, A_values, *, record_every=0, stream=None, **kw):
        """delta(t_m) of Eq. 8 for len(A_values) x R twin pairs at m =
        record_every, 2 record_every, ..., M (record_every = 0: t_M only).
        Returns (steps, array n_records x len(A_values) x R)."""
        M = int(M)
        k = M if record_every <= 0 else int(record_every)
        marks = list(range(k, M, k)) + [M]
        tw = self.twin_run(variant, M, R, A_values, stream=stream, **kw)
        try:
            out = []
            done = 0
            for m in marks:
                tw.steps(m - done)
                done = m
                out.append(tw.delta())
        finally:
            tw.close()
        nA = len(np.atleast_1d(A_values))
        return np.asarray(marks), np.stack(out).reshape(len(marks), nA, int(R))

    def relaxed_energy_grad(self, variant, M, window, x0_ptr, R, A, dt, c, energy_ptr,
                            grad_x0_ptr=None, grad_A_ptr=None, grad_dt_ptr=None,
                            ckpt_every=20, precision="fp32", stream=None):
        """gsb_relaxed_energy_grad on caller device buffers (raw pointers);
        precision "fp32" (SGEMMs on CUDA cores) or "bf16x3" (the products on
        the tensor cores, split bf16)."""
        prm = gsb_params()
        prm.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        prm.variant = VARIANT[variant] if isinstance(variant, str) else int(variant)
        prm.M = int(M)
        prm.R = int(R)
        prm.c = float(c)
        prm.dt = float(dt)
        A_arr = np.asarray(A, dtype=np.float32)
        keep = None
        if A_arr.ndim == 0:
            prm.A = float(A_arr)
        else:
            keep = np.ascontiguousarray(A_arr)
            prm.A_per_replica = _p(keep, ctypes.c_float)
        _check(lib().gsb_relaxed_energy_grad(self.handle, ctypes.byref(prm), int(window),
                                             int(ckpt_every), x0_ptr, energy_ptr, grad_x0_ptr,
                                             grad_A_ptr, grad_dt_ptr, _stream_handle(stream)))
        del keep

    def close(self):
        if self.handle:
            lib().gsb_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Run:
    """One GbSB / bSB / dSB run of R replicas over M steps (Sec. II)."""

    def __init__(self, problem, variant, M, R, *, c, dt, A, seed, precision, eval_every, x0, y0,
                 y0_uniform, x0_range, schedule, steps_per_launch, defer, profile, stream,
                 sm_pairs=False, fused_csr=False):
        self.problem = problem
        self.R = int(R)
        self.N = problem.N
        prm = gsb_params()
        prm.variant = VARIANT[variant] if isinstance(variant, str) else int(variant)
        prm.M = int(M)
        prm.R = int(R)
        prm.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        prm.c = float(c)
        prm.dt = float(dt)
        keep = []
        A_arr = np.asarray(A, dtype=np.float32)
        if A_arr.ndim == 0:
            prm.A = float(A_arr)
        else:
            a = np.ascontiguousarray(A_arr)
            keep.append(a)
            prm.A_per_replica = _p(a, ctypes.c_float)
        if schedule is not None:
            s = np.ascontiguousarray(schedule, dtype=np.float32)
            keep.append(s)
            prm.schedule = _p(s, ctypes.c_float)
        prm.seed = int(seed)
        prm.x0_range = float(x0_range)
        prm.y0_uniform = int(bool(y0_uniform))
        prm.eval_every = int(eval_every)
        prm.steps_per_launch = int(steps_per_launch)
        if x0 is not None:
            xa = np.ascontiguousarray(x0, dtype=np.float32)
            keep.append(xa)
            prm.x0 = _p(xa, ctypes.c_float)
        if y0 is not None:
            ya = np.ascontiguousarray(y0, dtype=np.float32)
            keep.append(ya)
            prm.y0 = _p(ya, ctypes.c_float)
        prm.flags = ((RUN_DEFER if defer else 0) | (RUN_PROFILE if profile else 0)
                     | (RUN_SM_PAIRS if sm_pairs else 0) | (RUN_FUSED_CSR if fused_csr else 0))
        out = _vp()
        _check(lib().gsb_run(problem.handle, ctypes.byref(prm), ctypes.byref(out),
                             _stream_handle(stream)))
        self.handle = out

    def steps(self, n):
        _check(lib().gsb_run_steps(self.handle, int(n)))

    def restart(self, seed, defer=False):
        _check(lib().gsb_run_restart(self.handle, int(seed), RUN_DEFER if defer else 0))

    def kernel(self):
        """Name of the step kernel this run selected."""
        return lib().gsb_run_kernel(self.handle).decode()

    def kernel_time(self):
        """(total ms, launches, steps covered) of the step kernel since the last (re)start."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        k = ctypes.c_int64()
        _check(lib().gsb_kernel_time(self.handle, ctypes.byref(ms), ctypes.byref(n),
                                     ctypes.byref(k)))
        return ms.value, n.value, k.value

    def best(self, out=None):
        """Best state per replica: dict of spins s (R x N int8), energies E, cuts
        and the step found. out: optional dict of preallocated host arrays with
        those keys (e.g. views of pinned memory) to fill instead."""
        if out is None:
            out = {"s": np.zeros((self.R, self.N), dtype=np.int8),
                   "E": np.zeros(self.R, dtype=np.float64),
                   "cut": np.zeros(self.R, dtype=np.float64),
                   "step": np.zeros(self.R, dtype=np.int32)}
        spins, e, cut, step = out["s"], out["E"], out["cut"], out["step"]
        for a, dt, shape in ((spins, np.int8, (self.R, self.N)), (e, np.float64, (self.R,)),
                             (cut, np.float64, (self.R,)), (step, np.int32, (self.R,))):
            if a.dtype != dt or a.shape != shape or not a.flags.c_contiguous:
                raise ValueError("best(out=...): wrong dtype, shape or layout")
        _check(lib().gsb_best(self.handle, _p(spins, ctypes.c_int8), _p(e, ctypes.c_double),
                              _p(cut, ctypes.c_double), _p(step, ctypes.c_int32)))
        return {"s": spins, "E": e, "cut": cut, "step": step}

    def state(self):
        """Current x, y, p (R x n_spins, host) and the steps done so far."""
        x = np.zeros((self.R, self._n_state()), dtype=np.float32)
        y = np.zeros_like(x)
        p = np.zeros_like(x)
        done = ctypes.c_int32()
        _check(lib().gsb_get_state(self.handle, _p(x, ctypes.c_float), _p(y, ctypes.c_float),
                                   _p(p, ctypes.c_float), ctypes.byref(done)))
        return {"x": x, "y": y, "p": p, "steps": done.value}

    def set_state(self, state, best=None):
        """Checkpoint / resume (gsb_run_set_state): state as returned by state()
        (x, y, p, steps), best as returned by best() or None."""
        x = np.ascontiguousarray(state["x"], dtype=np.float32)
        y = np.ascontiguousarray(state["y"], dtype=np.float32)
        p = None if state.get("p") is None else np.ascontiguousarray(state["p"], dtype=np.float32)
        s = e = k = None
        if best is not None:
            s = np.ascontiguousarray(best["s"], dtype=np.int8)
            e = np.ascontiguousarray(best["E"], dtype=np.float64)
            k = np.ascontiguousarray(best["step"], dtype=np.int32)
        _check(lib().gsb_run_set_state(self.handle, _p(x, ctypes.c_float), _p(y, ctypes.c_float),
                                       _p(p, ctypes.c_float), int(state["steps"]),
                                       _p(s, ctypes.c_int8), _p(e, ctypes.c_double),
                                       _p(k, ctypes.c_int32)))

    def _n_state(self):
        n = ctypes.c_int32()
        _check(lib().gsb_problem_info(self.problem.handle, ctypes.byref(n), None, None, None))
        return n.value

    def close(self):
        if self.handle:
            lib().gsb_run_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TwinRun(Run):
    """Twin trajectories of Sec. IV (gsb_twin_run): len(A_values) x R pairs;
    replica a R + r is trajectory (1) of pair (a, r), replica
    len(A_values) R + a R + r its trajectory (2)."""

    def __init__(self, problem, variant, M, R, A_values, *, c, dt, seed, precision, eval_every,
                 schedule, steps_per_launch, defer, profile, stream):
        self.problem = problem
        A = np.ascontiguousarray(np.atleast_1d(A_values), dtype=np.float32)
        self.pairs = len(A) * int(R)
        self.R = 2 * self.pairs
        self.N = problem.N
        prm = _make_params(variant, M, R, c=c, dt=dt, seed=seed, precision=precision,
                           eval_every=eval_every)
        keep = None
        if schedule is not None:
            keep = np.ascontiguousarray(schedule, dtype=np.float32)
            prm.schedule = _p(keep, ctypes.c_float)
        prm.steps_per_launch = int(steps_per_launch)
        prm.flags = (RUN_DEFER if defer else 0) | (RUN_PROFILE if profile else 0)
        out = _vp()
        _check(lib().gsb_twin_run(problem.handle, ctypes.byref(prm), len(A),
                                  _p(A, ctypes.c_float), ctypes.byref(out),
                                  _stream_handle(stream)))
        self.handle = out

    def delta(self):
        """Eq. 8 for every pair at the current step (host, FP64)."""
        out = np.zeros(self.pairs, dtype=np.float64)
        _check(lib().gsb_twin_delta(self.handle, _p(out, ctypes.c_double)))
        return out


_BatchRun.best = Run.best
_BatchRun.steps = Run.steps
_BatchRun.restart = Run.restart
_BatchRun.state = Run.state
_BatchRun._n_state = Run._n_state
_BatchRun.close = Run.close
_BatchRun.__del__ = Run.__del__
