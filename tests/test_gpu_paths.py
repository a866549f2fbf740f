"""Path selection on the GPU: the shapes the kernels were designed for must
take the fast forms, not a slower correct fallback."""
import math

import numpy as np
import pytest

from paper_2508_17655_gb300 import gsb, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build()


@pytest.mark.parametrize("variant", ["gdsb", "dsb"])
def test_k2000_shape_runs_the_persistent_fp8_kernel(variant):
    """N = 2000 (+-1 couplings), R = 1024 on the FP8 path runs the persistent
    kernel, one launch covering many steps: the cooperative grid form (the 8
    clusters of 16 CTAs of the cluster form would not all fit at once on a
    GB300, and a second wave would double the time; spin blocks of 112, 144
    CTAs, where they fit), or the cluster form where every cluster fits."""
    N, R, M = 2000, 1024, 2000
    P = gsb.Problem.dense(I.sk_pm1(N, 0))
    A = np.repeat(np.linspace(0.0, 0.35, 8).astype(np.float32), R // 8)
    run = P.run(variant, M=M, R=R, c=1 / (2 * math.sqrt(N)), dt=1.25, A=A, seed=1,
                precision="fp8", defer=True, profile=True)
    assert run.kernel() in ("k_tc_persist<grid112>", "k_tc_persist<grid>",
                            "k_tc_persist<cluster>")
    run.steps(64)
    ms, launches, steps = run.kernel_time()
    assert steps == 64
    assert launches < steps, f"{launches} launches for {steps} steps: per-step fallback"
