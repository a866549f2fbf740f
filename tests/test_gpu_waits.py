"""Failure detection without a GPU fault: a device-side wait that nothing
satisfies gives up after its time limit, the call returns GSB_ETIMEOUT, and the
CUDA context is still usable (a run afterwards matches the same run before)."""
import time

import numpy as np
import pytest

from paper_2508_17655_gb300 import gsb, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build()


def _small_run():
    P = gsb.Problem.dense(I.sk_pm1(300, 2))
    run = P.run("gdsb", M=200, R=256, c=0.03, dt=1.0, A=0.2, seed=4)
    b = run.best()
    run.close()
    P.close()
    return b


@pytest.mark.parametrize("kind", [0, 1])
def test_unsatisfied_wait_times_out_and_context_survives(kind):
    before = _small_run()
    t = time.perf_counter()
    with pytest.raises(gsb.GsbError) as e:
        gsb.wait_check(kind, 20_000_000)  # 20 ms of device time
    el = time.perf_counter() - t
    assert e.value.status == gsb.ETIMEOUT
    assert el < 2.0
    after = _small_run()
    np.testing.assert_array_equal(before["E"], after["E"])
    np.testing.assert_array_equal(before["s"], after["s"])


def test_satisfied_wait_returns_ok():
    gsb.wait_check(2, 20_000_000)


def test_wait_check_rejects_bad_arguments():
    with pytest.raises(gsb.GsbError) as e:
        gsb.wait_check(3, 20_000_000)
    assert e.value.status == gsb.EINVAL
    with pytest.raises(gsb.GsbError) as e:
        gsb.wait_check(0, 10)
    assert e.value.status == gsb.EINVAL
