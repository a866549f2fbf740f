"""Parameter sweeps of Fig. 1 and Fig. 5 on top of the run API.

* ``success_grid``: success probability P_S (with its 99 % interval), the
  average cut normalised by the best known cut (C_ave / C_best, Fig. 5) and
  TTS99 (Sec. VI) over an (M, A) grid, as in Fig. 1(a-c). All control
  strengths of one M run together in one launch sequence: replica
  k reps + r uses A_k (Eq. 7 keeps replicas independent).
* ``success_grid_dt``: the same over a (Delta_t, t_M) grid at fixed A, M =
  round(t_M / Delta_t), as in Fig. 1(g-i).
* ``delta_grid`` / ``delta_grid_dt``: the twin distance delta(t_M) of Eq. 8
  averaged over pairs (Sec. IV) on the same grids (Fig. 1(d-f), (j-l)).

Every run is an ordinary library run (or twin run); nothing here computes a
step. TTS takes as T_com the host wall time of the run that produced the
cell (all replicas of the run advance together), and the batch of the reps
replicas of a cell as one attempt: P_batch = 1 - (1 - P_S)^reps.
"""
import time

import numpy as np

from . import stats


def _wall(run, M):
    t = time.perf_counter()
    run.steps(M)
    best = run.best()  # blocks on the run's stream
    return best, time.perf_counter() - t


def _cells(best, As, reps, E_target, run_s, C_best):
    E = best["E"].reshape(len(As), reps)
    cut = best["cut"].reshape(len(As), reps)
    out = []
    for k in range(len(As)):
        succ = int(np.sum(E[k] <= E_target + 1e-9))
        ps, dps = stats.success_probability(succ, reps)
        pb = stats.batch_success(ps, reps)
        out.append({"P_S": ps, "P_S_err": dps, "P_S_ci99": stats.binomial_interval(succ, reps),
                    "mean_E": float(E[k].mean()), "min_E": float(E[k].min()),
                    "C_ave": float(cut[k].mean()), "max_cut": float(cut[k].max()),
                    "TTS99_s": stats.time_to_solution(pb, run_s)})
    return out


def _finish(cells, C_best):
    best_seen = max(c["max_cut"] for row in cells for c in row)
    cb = best_seen if C_best is None else float(C_best)
    for row in cells:
        for c in row:
            c["C_ave_over_C_best"] = c["C_ave"] / cb if cb else float("nan")
    return cb


def _table(cells, key):
    return np.array([[c[key] for c in row] for row in cells], dtype=np.float64)


def success_grid(problem, variant, Ms, As, reps, E_target, *, c=0.0, dt=0.0, seed=1,
                 precision="auto", C_best=None, stream=None):
    """P_S, C_ave / C_best and TTS99 on the (M, A) grid. C_best: the best
    known cut (default: the best cut any cell found). Returns a dict of
    len(Ms) x len(As) arrays plus the per-M run wall times."""
    As = [float(a) for a in As]
    A_rep = np.repeat(np.asarray(As, np.float32), reps)
    cells, times = [], []
    for M in Ms:
        run = problem.run(variant, M=int(M), R=len(As) * reps, c=c, dt=dt, A=A_rep, seed=seed,
                          precision=precision, defer=True, stream=stream)
        try:
            best, run_s = _wall(run, int(M))
        finally:
            run.close()
        cells.append(_cells(best, As, reps, E_target, run_s, C_best))
        times.append(run_s)
    cb = _finish(cells, C_best)
    return {"M": list(Ms), "A": As, "reps": reps, "E_target": E_target, "C_best": cb,
            "P_S": _table(cells, "P_S"), "P_S_err": _table(cells, "P_S_err"),
            "C_ave_over_C_best": _table(cells, "C_ave_over_C_best"),
            "mean_E": _table(cells, "mean_E"), "TTS99_s": _table(cells, "TTS99_s"),
            "run_s": np.asarray(times)}


def success_grid_dt(problem, variant, dts, tMs, A, reps, E_target, *, c=0.0, seed=1,
                    precision="auto", C_best=None, stream=None):
    """P_S, C_ave / C_best and TTS99 on the (Delta_t, t_M) grid at control
    strength A; M = max(1, round(t_M / Delta_t))."""
    cells, Ms = [], []
    for dt in dts:
        row, mrow = [], []
        for tM in tMs:
            M = max(1, int(round(tM / dt)))
            run = problem.run(variant, M=M, R=reps, c=c, dt=float(dt), A=float(A), seed=seed,
                              precision=precision, defer=True, stream=stream)
            try:
                best, run_s = _wall(run, M)
            finally:
                run.close()
            row.extend(_cells(best, [A], reps, E_target, run_s, C_best))
            mrow.append(M)
        cells.append(row)
        Ms.append(mrow)
    cb = _finish(cells, C_best)
    return {"dt": list(dts), "t_M": list(tMs), "A": float(A), "M": np.asarray(Ms), "reps": reps,
            "E_target": E_target, "C_best": cb, "P_S": _table(cells, "P_S"),
            "C_ave_over_C_best": _table(cells, "C_ave_over_C_best"),
            "mean_E": _table(cells, "mean_E"), "TTS99_s": _table(cells, "TTS99_s")}


def delta_grid(problem, variant, Ms, As, pairs, *, c=0.0, dt=0.0, seed=1, precision="auto",
               stream=None):
    """delta(t_M) of Eq. 8 on the (M, A) grid: all A of one M in one twin run;
    returns the per-cell mean over pairs and every pair's value."""
    mean, every = [], []
    for M in Ms:
        _, d = problem.twin_delta(variant, int(M), pairs, As, c=c, dt=dt, seed=seed,
                                  precision=precision, stream=stream)
        every.append(d[-1])
        mean.append(d[-1].mean(axis=1))
    return {"M": list(Ms), "A": [float(a) for a in As], "pairs": pairs,
            "delta_mean": np.asarray(mean), "delta": np.asarray(every)}


def delta_grid_dt(problem, variant, dts, tMs, A, pairs, *, c=0.0, seed=1, precision="auto",
                  stream=None):
    """delta(t_M) on the (Delta_t, t_M) grid at control strength A."""
    mean, Ms = [], []
    for dt in dts:
        row, mrow = [], []
        for tM in tMs:
            M = max(1, int(round(tM / dt)))
            _, d = problem.twin_delta(variant, M, pairs, [A], c=c, dt=float(dt), seed=seed,
                                      precision=precision, stream=stream)
            row.append(float(d[-1][0].mean()))
            mrow.append(M)
        mean.append(row)
        Ms.append(mrow)
    return {"dt": list(dts), "t_M": list(tMs), "A": float(A), "M": np.asarray(Ms),
            "pairs": pairs, "delta_mean": np.asarray(mean)}
