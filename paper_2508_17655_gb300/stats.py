"""Success statistics of a batch of runs (Sec. VI): success probability with an
exact binomial interval, time to solution and its error.

TTS is the time to find the target with 99 % probability by repeating a run
of time T_com that succeeds with probability P_S: T_com ln(1 - 0.99) /
ln(1 - P_S), or T_com itself once P_S exceeds 0.99. Its error follows from
Delta P_S = sqrt(P_S (1 - P_S) / N_rep) by propagation through the logarithm.
"""
import math


def success_probability(k, n):
    """P_S = k / n and its standard error sqrt(P_S (1 - P_S) / n)."""
    if n <= 0:
        raise ValueError("n must be positive")
    ps = k / n
    return ps, math.sqrt(max(ps * (1.0 - ps), 0.0) / n)


def binomial_interval(k, n, conf=0.99):
    """Exact (Clopper-Pearson) interval for a binomial proportion: the bounds
    are the quantiles alpha/2 of Beta(k, n - k + 1) and 1 - alpha/2 of
    Beta(k + 1, n - k), taken from the inverse regularised incomplete beta
    function."""
    from scipy.special import betaincinv
    if not 0 <= k <= n or n <= 0:
        raise ValueError("need 0 <= k <= n, n > 0")
    alpha = 1.0 - conf
    lo = 0.0 if k == 0 else float(betaincinv(k, n - k + 1, alpha / 2))
    hi = 1.0 if k == n else float(betaincinv(k + 1, n - k, 1.0 - alpha / 2))
    return lo, hi


def time_to_solution(ps, t_com, target=0.99):
    """TTS for success probability ps per run of duration t_com (inf at ps = 0)."""
    if ps >= 1.0 or ps > target:
        return t_com
    if ps <= 0.0:
        return math.inf
    return t_com * math.log1p(-target) / math.log1p(-ps)


def time_to_solution_error(ps, t_com, nrep, target=0.99):
    """Delta TTS = TTS Delta P_S / ((1 - P_S) |ln(1 - P_S)|); zero where TTS is
    t_com itself, inf where TTS is."""
    t = time_to_solution(ps, t_com, target)
    if not math.isfinite(t):
        return math.inf
    if ps >= 1.0 or ps > target:
        return 0.0
    _, dps = success_probability(ps * nrep, nrep)
    return t * dps / ((1.0 - ps) * abs(math.log1p(-ps)))


def batch_success(ps, batch):
    """Success probability of a batch of independent runs (any of them succeeds)."""
    return 1.0 - (1.0 - ps) ** batch
