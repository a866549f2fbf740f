"""The sweep harness on the GPU: every cell of an (M, A) success grid is the
slice of one ordinary run (same energies, replica for replica, as a direct
gsb_run with the same per-replica control strengths and seed), and the
delta grid equals direct twin runs."""
import numpy as np
import pytest

from paper_2508_17655_gb300 import gsb, inputs as I, stats, sweep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build()


def test_success_grid_cells_are_slices_of_direct_runs():
    N, reps, As, Ms = 100, 64, [0.0, 0.2, 0.4], [150, 300]
    J = I.sk_pm1(N, 0)
    P = gsb.Problem.dense(J)
    E_target = -600.0
    g = sweep.success_grid(P, "gbsb", Ms, As, reps, E_target, c=0.05, dt=0.5, seed=9)
    for i, M in enumerate(Ms):
        A_rep = np.repeat(np.float32(As), reps)
        run = P.run("gbsb", M=M, R=len(As) * reps, c=0.05, dt=0.5, A=A_rep, seed=9)
        E = run.best()["E"].reshape(len(As), reps)
        run.close()
        for k in range(len(As)):
            succ = int(np.sum(E[k] <= E_target + 1e-9))
            assert g["P_S"][i, k] == succ / reps
            assert g["mean_E"][i, k] == E[k].mean()
    assert np.all(g["C_ave_over_C_best"] <= 1.0) and np.all(g["C_ave_over_C_best"] > 0.5)


def test_delta_grid_equals_twin_runs():
    N, pairs, As, Ms = 120, 32, [0.0, 0.8], [100, 200]
    J = I.sk_pm1(N, 1)
    P = gsb.Problem.dense(J)
    g = sweep.delta_grid(P, "gbsb", Ms, As, pairs, c=0.05, dt=0.5, seed=4)
    for i, M in enumerate(Ms):
        _, d = P.twin_delta("gbsb", M, pairs, As, c=0.05, dt=0.5, seed=4)
        np.testing.assert_array_equal(g["delta"][i], d[-1])
        np.testing.assert_array_equal(g["delta_mean"][i], d[-1].mean(axis=1))


def test_delta_grid_dt_equals_twin_runs():
    """The (dt, t_M) grid of Fig. 1(j): each cell is a twin run with
    M = round(t_M / dt) steps, its mean distance that run's."""
    N, pairs = 120, 24
    J = I.sk_pm1(N, 2)
    P = gsb.Problem.dense(J)
    dts, tMs = [0.5, 1.25], [25.0, 60.0]
    g = sweep.delta_grid_dt(P, "gbsb", dts, tMs, 0.3, pairs, c=0.05, seed=8)
    assert g["M"].tolist() == [[50, 120], [20, 48]]
    for a, dt in enumerate(dts):
        for b, tM in enumerate(tMs):
            M = int(round(tM / dt))
            _, d = P.twin_delta("gbsb", M, pairs, [0.3], c=0.05, dt=dt, seed=8)
            assert g["delta_mean"][a, b] == float(d[-1][0].mean())


def test_success_grid_dt_cells_are_runs():
    N, reps = 100, 64
    J = I.sk_pm1(N, 0)
    P = gsb.Problem.dense(J)
    dts, tMs = [0.5, 1.0], [100.0]
    g = sweep.success_grid_dt(P, "gdsb", dts, tMs, 0.2, reps, -600.0, c=0.05, seed=3)
    for a, dt in enumerate(dts):
        M = int(round(100.0 / dt))
        run = P.run("gdsb", M=M, R=reps, c=0.05, dt=dt, A=0.2, seed=3)
        E = run.best()["E"]
        run.close()
        assert g["mean_E"][a, 0] == pytest.approx(float(E.mean()), rel=1e-14)
        assert g["P_S"][a, 0] == float(np.mean(E <= -600.0 + 1e-9))
