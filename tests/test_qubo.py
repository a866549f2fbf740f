"""QUBO input (gsb_qubo_to_ising / gsb_create_qubo): minimise f(b) = b^T Q b over
b in {0,1}^N through the Ising form of Eq. 1 with s = 2b - 1.

CPU: the library's host-side map is checked against the QUBO definition by
enumerating every b (brute force) and against the oracle's Gray-code ground
state of the equivalent Ising problem. GPU: a run on a QUBO problem reports
energies that map back to f(b) of the spins it returns, exactly, and finds
the brute-force minimum of a small instance."""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2508_17655_gb300 import build as B


@pytest.fixture(scope="module")
def gsb():
    B.build()
    from paper_2508_17655_gb300 import gsb as G
    return G


def _qubo(N, seed, lo=-5, hi=5):
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(N, N)).astype(np.float32)  # asymmetric, with diagonal


def _all_b(N):
    return np.array(list(itertools.product((0, 1), repeat=N)), dtype=np.float64)


def _f(Q, b):
    """The QUBO objective as defined: sum_ij Q_ij b_i b_j (rows of b)."""
    Q = np.asarray(Q, dtype=np.float64)
    return np.einsum("ki,ij,kj->k", b, Q, b)


@pytest.mark.parametrize("N,seed", [(1, 0), (2, 1), (7, 2), (12, 3)])
def test_qubo_map_reproduces_f_on_every_state(gsb, N, seed):
    Q = _qubo(N, seed)
    J, h, scale, offset = gsb.qubo_to_ising(Q)
    assert scale == 0.25
    np.testing.assert_array_equal(J, J.T)
    assert np.all(np.diag(J) == 0)
    assert np.all(J == np.round(J)) and np.all(h == np.round(h))  # integer Q -> integer J, h
    b = _all_b(N)
    s = 2 * b - 1
    E = -0.5 * np.einsum("ki,ij,kj->k", s, J.astype(np.float64), s) - s @ h.astype(np.float64)
    np.testing.assert_array_equal(scale * E + offset, _f(Q, b))


@pytest.mark.parametrize("N,seed", [(9, 4), (13, 5)])
def test_qubo_minimum_equals_oracle_ising_ground_state(gsb, N, seed):
    """min_b f(b) by enumeration = scale * (oracle Gray-code ground energy of the
    Ising problem, local field folded in as an extra spin) + offset."""
    Q = _qubo(N, seed)
    J, h, scale, offset = gsb.qubo_to_ising(Q)
    Ja = np.zeros((N + 1, N + 1))
    Ja[:N, :N] = J
    Ja[:N, N] = Ja[N, :N] = h
    e_min, s_min = O.bruteforce(Ja)
    fmin = _f(Q, _all_b(N)).min()
    assert scale * e_min + offset == fmin
    g = 1 if s_min[N] > 0 else -1  # gauge-fix the auxiliary spin to +1
    b = (1 + g * s_min[:N].astype(np.float64)) / 2
    assert _f(Q, b[None])[0] == fmin


def test_qubo_map_rejects_bad_input(gsb):
    Q = np.ones((3, 3), dtype=np.float32)
    Q[1, 2] = np.nan
    with pytest.raises(gsb.GsbError) as e:
        gsb.qubo_to_ising(Q)
    assert e.value.status == gsb.EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("variant", ["gbsb", "gdsb"])
def test_gpu_qubo_run_maps_back_and_finds_minimum(gsb, variant):
    N = 14
    Q = _qubo(N, 6)
    P = gsb.Problem.qubo(Q)
    fmin = _f(Q, _all_b(N)).min()
    r = P.run(variant, 1000, 256, A=0.2, seed=3)
    best = r.best()
    b = (1 + best["s"].astype(np.float64)) / 2
    # every reported energy is the Ising energy of the reported spins: mapped
    # back, it is exactly f(b)
    np.testing.assert_array_equal(P.scale * best["E"] + P.offset, _f(Q, b))
    assert (P.scale * best["E"] + P.offset).min() == fmin
    r.close()
    P.close()
