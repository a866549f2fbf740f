"""Host-side checks of a CSR coupling matrix through the C ABI, without a GPU:
a corrupt matrix is rejected with GSB_EINVAL and a message before the library
touches the device (rowptr bounds and monotonicity, column range and order,
symmetry, zero diagonal, finite values)."""
import ctypes

import numpy as np
import pytest

from paper_2508_17655_gb300 import gsb, inputs as I


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build()


def _create(N, rp, col, val, flags=0):
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float32)
    out = ctypes.c_void_p()
    st = gsb.lib().gsb_create(ctypes.byref(out), N, gsb.J_CSR_F32, None,
                              rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                              col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                              val.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(col), None,
                              flags, None)
    if st == gsb.OK:
        gsb.lib().gsb_destroy(out)
    return st, gsb.lib().gsb_last_error().decode()


def _good(N=40):
    return I.er_graph(N, 6, "pm1", 3)


def test_valid_matrix_passes_the_host_checks():
    rp, col, val = _good()
    st, _ = _create(40, rp, col, val)
    assert st in (gsb.OK, gsb.ENODEV, gsb.ECUDA)  # no GPU here: stops at the device check


@pytest.mark.parametrize("corruption,needle", [
    ("rowptr_start", "rowptr must run"),
    ("rowptr_end", "rowptr must run"),
    ("rowptr_order", "not monotone"),
    ("col_range", "out of range"),
    ("col_order", "must increase"),
    ("asymmetric", "not symmetric"),
    ("diagonal", "diagonal"),
    ("nan", "non-finite"),
])
def test_corrupt_matrix_is_rejected_on_the_host(corruption, needle):
    N = 40
    rp, col, val = (np.array(a) for a in _good(N))
    if corruption == "rowptr_start":
        rp[0] = 1
    elif corruption == "rowptr_end":
        rp[-1] -= 1
    elif corruption == "rowptr_order":
        i = int(np.argmax(np.diff(rp) >= 2))  # a row with two entries or more
        rp[i + 1] = rp[i] - 1 if rp[i] > 0 else rp[i + 2] + 1
    elif corruption == "col_range":
        col[3] = N + 5
    elif corruption == "col_order":
        i = int(np.argmax(np.diff(rp) >= 2))
        k = rp[i]
        col[k], col[k + 1] = col[k + 1], col[k]
    elif corruption == "asymmetric":
        val[5] = -val[5]
    elif corruption == "diagonal":
        # put J_00 on row 0 (column 0 comes first in a sorted row)
        col = np.concatenate([[0], col])
        val = np.concatenate([[1.0], val])
        rp = rp + 1
        rp[0] = 0
    elif corruption == "nan":
        val[7] = np.nan
    st, msg = _create(N, rp, col, val)
    assert st == gsb.EINVAL, (st, msg)
    assert needle in msg, msg


def test_unvalidated_creation_still_checks_structure():
    N = 40
    rp, col, val = (np.array(a) for a in _good(N))
    val[5] = -val[5]  # asymmetric values pass without validation
    st, _ = _create(N, rp, col, val, flags=gsb.CREATE_NO_VALIDATE)
    assert st in (gsb.OK, gsb.ENODEV, gsb.ECUDA)
    col[3] = N + 1  # but an index out of range never does
    st, msg = _create(N, rp, col, val, flags=gsb.CREATE_NO_VALIDATE)
    assert st == gsb.EINVAL and "out of range" in msg
