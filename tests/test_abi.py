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


C_CALLER = r"""
#include <stdio.h>
#include <string.h>
#include "gsb.h"

/* A plain C99 caller: only C types cross the boundary. No GPU work: every call
   below is rejected or answered before the library touches the device. */
int main(void) {
    gsb_problem* P = (gsb_problem*)1;
    gsb_params prm;
    memset(&prm, 0, sizeof prm);
    if (gsb_version() < 100) return 1;
    if (gsb_launch_count() < 0) return 2;
    if (gsb_create(&P, 0, GSB_J_DENSE_I8, NULL, NULL, NULL, NULL, 0, NULL, 0, NULL) != GSB_EINVAL)
        return 3;
    if (P != NULL) return 4;                         /* *out cleared on failure */
    if (strlen(gsb_last_error()) == 0) return 5;     /* a message for the failure */
    if (gsb_run(NULL, &prm, NULL, NULL) != GSB_EINVAL) return 6;
    if (gsb_run_destroy(NULL) != GSB_OK) return 7;
    if (gsb_twin_delta(NULL, NULL) != GSB_EINVAL) return 8;
    if (gsb_wait_check(7, 1000000, NULL) != GSB_EINVAL) return 9;
    if (strcmp(gsb_run_kernel(NULL), "") != 0) return 10;
    if (gsb_release_cached_memory() != GSB_OK) return 11;  /* nothing kept yet */
    if (gsb_set_memory_limit(-1) != GSB_EINVAL) return 12;
    if (gsb_set_memory_limit(0) != GSB_OK) return 13;
    {
        int64_t used = -1, kept = -1;
        if (gsb_memory_usage(&used, &kept) != GSB_OK || used != 0 || kept != 0) return 14;
    }
    printf("ok\n");
    return 0;
}
"""


def test_plain_c_caller_compiles_links_and_runs(libpath, tmp_path):
    """include/gsb.h is a C header (gcc -std=c99 -Wall -Werror), the library
    links from C, and argument errors come back as statuses with a message."""
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(libpath)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                        "-L", libdir, "-l:" + os.path.basename(libpath),
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0 and run.stdout.strip() == "ok", (run.returncode, run.stderr)
