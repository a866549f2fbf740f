"""The debug build (-DGSB_DEBUG) on the GPU. Its kernels check on the device
the indices that come from the caller's data (CSR row ranges and columns,
batched tile lists) and their launch geometry; a failed check skips the access
and sets a bit in the status word, so nothing traps. Here:

* the checks fire: gsb_debug_selftest plants an out-of-range CSR column and a
  tensor-core launch one spin block too tall, and both are caught without the
  access; a run afterwards works (the context survives);
* on valid inputs no check fires and the results are the release build's, bit
  for bit, over every path (dense FP8 persistent and per-step, FX32, FX16, split
  bf16, FP32, CSR per-step and fused, batched in both forms, Lyapunov and
  adjoint in both coupling forms) at the tiling's edge sizes (N = 1, 2, 17,
  127, 129; R = 1, 3, 130; 134 replicas with tangents).

The debug library runs in a child process (GSB_LIBRARY=debug); the release
results come from this process."""
import os
import subprocess
import sys

import numpy as np
import pytest

from tests import _debug_cases as C

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _child(args, timeout=900):
    env = dict(os.environ, GSB_LIBRARY="debug")
    r = subprocess.run([sys.executable, *args], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=timeout)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return r.stdout


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build_all()


def test_debug_checks_fire_without_faulting():
    out = _child(["-c", (
        "from paper_2508_17655_gb300 import gsb, inputs as I\n"
        "assert gsb.debug_build()\n"
        "gsb.debug_selftest()\n"
        "gsb.debug_selftest()\n"
        "P = gsb.Problem.dense(I.sk_pm1(300, 1))\n"
        "b = P.run('gdsb', M=40, R=130, c=0.03, dt=1.0, A=0.2, seed=3).best()\n"
        "print('ok', len(b['E']))\n")])
    assert "ok 130" in out


def test_debug_build_matches_release_bit_exact(tmp_path):
    from paper_2508_17655_gb300 import gsb
    assert not gsb.debug_build()
    path = tmp_path / "debug.npz"
    _child([os.path.join("tests", "_debug_cases.py"), str(path)])
    dbg = dict(np.load(path))
    assert int(dbg.pop("debug_build")) == 1
    rel = C.run_cases()
    assert len(rel) == len(dbg)
    for k, v in rel.items():
        np.testing.assert_array_equal(dbg[k.replace("/", "|")], v, err_msg=k)
