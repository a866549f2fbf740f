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


def test_reused_device_blocks_give_identical_runs():
    """Problems and runs created again with the same shape take the blocks the
    destroyed ones left (no cudaMalloc); whatever those blocks held, the new run
    follows the same trajectory (every buffer the step kernels read is written
    first), on the FP8, FX32, FP32 and CSR paths, and after the cache is
    returned to CUDA."""
    def once(kind):
        if kind == "csr":
            rp, col, val = I.er_graph(300, 12, "pm1", 2)
            P = gsb.Problem.csr(300, rp, col, val)
            run = P.run("gdsb", M=120, R=200, c=0.05, dt=0.8, A=0.3, seed=6, eval_every=40)
        else:
            variant, prec = {"fp8": ("gdsb", "fp8"), "fx32": ("gbsb", "fx32"),
                             "fp32": ("gbsb", "fp32")}[kind]
            P = gsb.Problem.dense(I.sk_pm1(300, 2))
            run = P.run(variant, M=120, R=200, c=0.03, dt=1.0, A=0.3, seed=6, precision=prec,
                        eval_every=40)
        b, st = run.best(), run.state()
        run.close()
        P.close()
        return b, st
    for kind in ("fp8", "fx32", "fp32", "csr"):
        first = once(kind)
        again = once(kind)
        for k in ("E", "s", "step"):
            np.testing.assert_array_equal(first[0][k], again[0][k])
        for k in ("x", "y", "p"):
            np.testing.assert_array_equal(first[1][k], again[1][k])
    gsb.release_cached_memory()
    after = once("fp8")
    np.testing.assert_array_equal(after[0]["E"], once("fp8")[0]["E"])


def test_memory_limit_gives_enomem_and_leaves_nothing_behind():
    """Failure detection on the host: a cap on the library's device memory makes
    an allocation fail; the call returns GSB_ENOMEM with a message and releases
    what it had taken; with the cap lifted the same call succeeds."""
    import gc
    gc.collect()  # handles of earlier tests freed now, not during this one
    gsb.release_cached_memory()
    used0, _ = gsb.memory_usage()
    try:
        gsb.set_memory_limit(used0 + (1 << 20))  # 1 MiB of headroom
        with pytest.raises(gsb.GsbError) as e:
            gsb.Problem.dense(I.sk_pm1(2000, 0))  # 16 MB of FP32 J alone
        assert e.value.status == gsb.ENOMEM
        assert gsb.memory_usage()[0] == used0
        P = gsb.Problem.dense(I.sk_pm1(64, 0))  # well inside the cap
        used1, _ = gsb.memory_usage()
        with pytest.raises(gsb.GsbError) as e:
            P.run("gdsb", M=10, R=65536, c=0.1, dt=1.0)
        assert e.value.status == gsb.ENOMEM
        assert gsb.memory_usage()[0] == used1
    finally:
        gsb.set_memory_limit(0)
    run = P.run("gdsb", M=10, R=65536, c=0.1, dt=1.0)
    assert np.all(np.isfinite(run.best()["E"]))
    run.close()
    P.close()
    assert gsb.memory_usage()[0] == used0
