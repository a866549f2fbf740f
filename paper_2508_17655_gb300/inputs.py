"""Seeded synthetic instances shaped like the paper's workloads.

This module holds only input generation (no part of the method's arithmetic);
the tests, the benchmark and the oracle all take their couplings from here.

* ``sk_pm1``: complete graph with i.i.d. +-1 couplings, symmetric, zero
  diagonal -- the shape of K2000 and of the 700-spin instances (Sec. III).
* ``sk_gauss``: Sherrington-Kirkpatrick couplings N(0, 1/N).
* ``er_graph``: Erdos-Renyi graph with a given mean degree, unit (+1) or random
  +-1 edge weights W, stored as J = -W in CSR (G-set-like sparse Max-Cut,
  Sec. III: J in {0, -1} or {0, +-1}).
* ``ring`` / ``complete``: graphs whose maximum cut is known in closed form.
* ``batch_sizes``: sizes of a batch of uneven instances.
* ``uniform_state``: an explicit initial state, uniform in [-0.1, 0.1).
"""
from __future__ import annotations

import numpy as np


def sk_pm1(N: int, seed: int = 0) -> np.ndarray:
    """Symmetric N x N int8 matrix, i.i.d. +-1 above the diagonal, zero diagonal."""
    rng = np.random.default_rng(seed)
    U = rng.integers(0, 2, size=(N, N), dtype=np.int8) * 2 - 1
    J = np.triu(U, 1)
    J = (J + J.T).astype(np.int8)
    return J


def sk_gauss(N: int, seed: int = 0) -> np.ndarray:
    """Symmetric N x N float32 matrix, i.i.d. N(0, 1/N) above the diagonal."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal(size=(N, N)) / np.sqrt(N)
    J = np.triu(G, 1)
    return (J + J.T).astype(np.float32)


def er_edges(N: int, mean_degree: float, seed: int = 0):
    """Edge list (i < j) of a G(N, m) graph with m = round(mean_degree N / 2)."""
    rng = np.random.default_rng(seed)
    m = int(round(mean_degree * N / 2))
    total = N * (N - 1) // 2
    m = min(m, total)
    chosen = set()
    out_i, out_j = [], []
    while len(out_i) < m:
        need = m - len(out_i)
        a = rng.integers(0, N, size=2 * need + 16)
        b = rng.integers(0, N, size=2 * need + 16)
        for u, v in zip(a.tolist(), b.tolist()):
            if u == v:
                continue
            i, j = (u, v) if u < v else (v, u)
            key = i * N + j
            if key in chosen:
                continue
            chosen.add(key)
            out_i.append(i)
            out_j.append(j)
            if len(out_i) == m:
                break
    return np.array(out_i, dtype=np.int64), np.array(out_j, dtype=np.int64)


def edges_to_csr(N: int, ei, ej, w):
    """Symmetric CSR of J = -W from an undirected weighted edge list."""
    rows = np.concatenate([ei, ej])
    cols = np.concatenate([ej, ei])
    vals = -np.concatenate([w, w]).astype(np.float32)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(N + 1, dtype=np.int32)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    return rowptr, cols.astype(np.int32), vals


def er_graph(N: int, mean_degree: float = 20.0, weights: str = "+1", seed: int = 0):
    """Erdos-Renyi Max-Cut instance as CSR (rowptr, col, val) of J = -W.

    weights: "+1" (all W = 1, J in {0, -1}) or "pm1" (W = +-1, J in {0, +-1})."""
    ei, ej = er_edges(N, mean_degree, seed)
    if weights == "+1":
        w = np.ones(len(ei), dtype=np.float32)
    elif weights == "pm1":
        rng = np.random.default_rng(seed + 7919)
        w = (rng.integers(0, 2, size=len(ei)) * 2 - 1).astype(np.float32)
    else:
        raise ValueError(weights)
    return edges_to_csr(N, ei, ej, w)


def csr_to_dense(N, rowptr, col, val):
    D = np.zeros((N, N), dtype=np.float64)
    for i in range(N):
        for k in range(rowptr[i], rowptr[i + 1]):
            D[i, col[k]] += val[k]
    return D


def ring(N: int, w: float = 1.0) -> np.ndarray:
    """Cycle graph C_N with edge weight w, as J = -W (dense)."""
    J = np.zeros((N, N), dtype=np.float64)
    for i in range(N):
        j = (i + 1) % N
        J[i, j] = J[j, i] = -w
    return J


def complete(N: int, w: float = 1.0) -> np.ndarray:
    """Complete graph K_N with edge weight w, as J = -W (dense)."""
    J = np.full((N, N), -w, dtype=np.float64)
    np.fill_diagonal(J, 0.0)
    return J


def batch_sizes(n: int, seed: int = 0, nmin: int = 64, nmax: int = 1024,
                rmin: int = 32, rmax: int = 256):
    """Sizes (N_k, R_k) of n uneven SK instances, N_k ~ U{nmin..nmax}, R_k ~ U{rmin..rmax}."""
    rng = np.random.default_rng(seed)
    Ns = rng.integers(nmin, nmax + 1, size=n)
    Rs = rng.integers(rmin, rmax + 1, size=n)
    return Ns.astype(np.int64), Rs.astype(np.int64)


def uniform_state(R: int, N: int, seed: int = 0, rng: float = 0.1) -> np.ndarray:
    """R x N float32 positions drawn i.i.d. uniform in [-rng, rng) (the range of
    x(0), App. A), for callers that hand the library an explicit initial state."""
    g = np.random.default_rng(seed)
    return g.uniform(-rng, rng, size=(R, N)).astype(np.float32)
