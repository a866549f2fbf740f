"""CPU-side checks of the debug build (-DGSB_DEBUG: device-side bounds checks
that report into the run's status word): it builds for sm_103a beside the
release library, exports every entry point include/gsb.h declares, and each
build reports what it is. gsb_debug_selftest of the release build refuses on
the host, launching nothing. No GPU is needed."""
import ctypes
import re
import subprocess

import pytest

from paper_2508_17655_gb300 import build as B
from tests.test_abi import declared_symbols

GSB_EUNSUPPORTED = 5


@pytest.fixture(scope="module")
def libs():
    return B.build(), B.build(debug=True)


def test_debug_library_exports_every_declared_symbol(libs):
    _, dbg = libs
    out = subprocess.run(["nm", "-D", "--defined-only", dbg], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (gsb_\w+)", out))
    names = declared_symbols()
    assert {"gsb_debug_build", "gsb_debug_selftest"} <= names
    assert names <= exported, sorted(names - exported)


def test_each_build_reports_what_it_is(libs):
    rel, dbg = (ctypes.CDLL(p) for p in libs)
    for L in (rel, dbg):
        L.gsb_debug_build.restype = ctypes.c_int32
        L.gsb_debug_selftest.restype = ctypes.c_int
    assert rel.gsb_debug_build() == 0
    assert dbg.gsb_debug_build() == 1
    assert rel.gsb_debug_selftest() == GSB_EUNSUPPORTED
