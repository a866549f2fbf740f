"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point include/gsb.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2508_17655_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gsb_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_library_exports_every_declared_symbol(libpath):
    names = declared_symbols()
    assert {"gsb_create", "gsb_run", "gsb_best", "gsb_energy"} <= names
    L = ctypes.CDLL(libpath)
    for n in sorted(names):
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (gsb_\w+)", out))
    assert names <= exported


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2508_17655_gb300 import gsb
    monkeypatch.setattr(gsb._build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gsb, "_LIB", None)
    with pytest.raises(RuntimeError, match="not built"):
        gsb.lib()


def test_version_and_launch_counter_without_gpu(libpath):
    from paper_2508_17655_gb300 import gsb
    L = gsb.lib()
    assert L.gsb_version() >= 100
    assert L.gsb_launch_count() >= 0
