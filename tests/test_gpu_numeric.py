"""Failure detection for a non-finite state (GSB_ENUMERIC), injected from the
host: a NaN placed in one oscillator's x(0), or written into a saved state
with gsb_run_set_state, propagates through Eqs. 3-4 (the wall test of Eq. 5
never fires on a NaN) and is reported when the next energy evaluation reads
the state. Nothing faults: the kernels only compute with the value. The
context stays usable, and a clean run afterwards is unaffected."""
import numpy as np
import pytest

import oracle as O
from paper_2508_17655_gb300 import gsb, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build()


CASES = [  # (variant, precision, kind): every step-kernel family
    ("gdsb", "fp8", "dense"),
    ("gbsb", "fx32", "dense"),
    ("gbsb", "fp32", "dense"),
    ("dsb", "auto", "csr"),
]


def _problem(kind, N):
    if kind == "csr":
        rp, col, val = I.er_graph(N, 10, "pm1", 2)
        return gsb.Problem.csr(N, rp, col, val)
    return gsb.Problem.dense(I.sk_pm1(N, 2))


@pytest.mark.parametrize("variant,precision,kind", CASES)
def test_nan_in_initial_state_reports_enumeric(variant, precision, kind):
    N, R, M = 300, 130, 20
    P = _problem(kind, N)
    x0 = O.init_uniform(R, N, 5).astype(np.float32)
    x0[7, 123] = np.nan
    run = P.run(variant, M, R, c=0.03, dt=0.5, A=0.2, x0=x0, precision=precision)
    with pytest.raises(gsb.GsbError) as e:
        run.best()
    assert e.value.status == gsb.ENUMERIC
    run.close()
    # the same problem runs cleanly afterwards: finite energies, each the
    # oracle's energy (Eq. 1) of the spins reported with it
    x0[7, 123] = 0.05
    ok = P.run(variant, M, R, c=0.03, dt=0.5, A=0.2, x0=x0, precision=precision).best()
    assert np.all(np.isfinite(ok["E"]))
    if kind == "csr":
        rp, col, val = I.er_graph(N, 10, "pm1", 2)
        Jo = O.Coupling(N, rowptr=rp, col=col, val=val)
    else:
        Jo = I.sk_pm1(N, 2).astype(np.float64)
    np.testing.assert_array_equal(ok["E"], O.energy(Jo, ok["s"]))


@pytest.mark.parametrize("variant,precision,kind", CASES[:2])
def test_nan_written_by_set_state_reports_enumeric(variant, precision, kind):
    N, R, M = 300, 130, 40
    P = _problem(kind, N)
    run = P.run(variant, M, R, c=0.03, dt=0.5, A=0.2, seed=4, precision=precision, defer=True)
    run.steps(10)
    st = run.state()
    st["x"][3, 17] = np.nan
    run.set_state(st)
    run.steps(M - 10)
    with pytest.raises(gsb.GsbError) as e:
        run.best()
    assert e.value.status == gsb.ENUMERIC
