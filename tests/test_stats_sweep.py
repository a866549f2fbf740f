"""Host logic of the success statistics (Sec. VI) and of the parameter-sweep
harness (Fig. 1, Fig. 5), without a GPU: the package's P_S interval and TTS
against the oracle's pinned formulas, and the sweep's bookkeeping on a fake
problem whose runs return known energies."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2508_17655_gb300 import stats, sweep


@pytest.mark.parametrize("k,n", [(0, 10), (1, 10), (5, 10), (10, 10), (7, 1000), (512, 1024)])
def test_binomial_interval_matches_oracle(k, n):
    lo, hi = stats.binomial_interval(k, n, 0.99)
    olo, ohi = O.clopper_pearson(k, n, 0.99)
    assert lo == pytest.approx(olo, rel=1e-9, abs=1e-15)
    assert hi == pytest.approx(ohi, rel=1e-9, abs=1e-15)
    assert lo <= k / n <= hi


@pytest.mark.parametrize("ps", [0.0, 1e-4, 0.013, 0.5, 0.98, 0.995, 1.0])
def test_tts_matches_oracle(ps):
    assert stats.time_to_solution(ps, 0.25) == O.tts(ps, 0.25) or (
        math.isfinite(O.tts(ps, 0.25)) and
        stats.time_to_solution(ps, 0.25) == pytest.approx(O.tts(ps, 0.25), rel=1e-12))
    e, eo = stats.time_to_solution_error(ps, 0.25, 1000), O.tts_error(ps, 0.25, 1000)
    assert (e == eo) or e == pytest.approx(eo, rel=1e-12)


def test_batch_success():
    assert stats.batch_success(0.0, 128) == 0.0
    assert stats.batch_success(1.0, 3) == 1.0
    assert stats.batch_success(0.5, 2) == pytest.approx(0.75)


class _FakeRun:
    def __init__(self, E, cut):
        self.E, self.cut, self.done = E, cut, 0

    def steps(self, n):
        self.done += n

    def best(self):
        return {"E": self.E, "cut": self.cut}

    def close(self):
        pass


class _FakeProblem:
    """run() returns energies -M - 10 k - r for replica k reps + r (A index k)."""

    def __init__(self):
        self.calls = []

    def run(self, variant, M, R, **kw):
        self.calls.append((M, R, kw))
        A = np.broadcast_to(np.asarray(kw["A"], np.float32), (R,))
        _, k = np.unique(A, return_inverse=True)  # control strength index
        r = np.arange(R) - np.searchsorted(A, A)  # position inside its group
        E = -(M + 10.0 * k + r)
        return _FakeRun(E, -E / 2)


def test_success_grid_bookkeeping():
    P = _FakeProblem()
    g = sweep.success_grid(P, "gbsb", [100, 200], [0.0, 0.1, 0.2], 4, E_target=-221.0)
    assert [c[1] for c in P.calls] == [12, 12]
    np.testing.assert_array_equal(P.calls[0][2]["A"], np.repeat(np.float32([0.0, 0.1, 0.2]), 4))
    # M = 200, A index 2: energies -220 .. -223, three of them <= -221
    assert g["P_S"][1, 2] == 0.75 and g["P_S"][0, 2] == 0.0 and g["P_S"][1, 1] == 0.0
    assert g["mean_E"][1, 2] == -221.5
    assert g["C_best"] == 223.0 / 2
    assert g["C_ave_over_C_best"][1, 2] == pytest.approx((221.5 / 2) / (223.0 / 2))
    assert math.isinf(g["TTS99_s"][0, 0]) and math.isfinite(g["TTS99_s"][1, 2])


def test_success_grid_dt_steps():
    P = _FakeProblem()
    g = sweep.success_grid_dt(P, "gbsb", [0.5, 1.25], [100.0, 250.0], 0.2, 2, E_target=0.0,
                              C_best=1000.0)
    assert g["M"].tolist() == [[200, 500], [80, 200]]
    assert [c[0] for c in P.calls] == [200, 500, 80, 200]
    assert np.all(g["P_S"] == 1.0) and g["C_best"] == 1000.0
