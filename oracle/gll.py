"""Legendre polynomials and Gauss-Lobatto-Legendre points (oracle; test infrastructure).

Overview (i) of the paper: the Lagrange basis lives on n+1 representation
points, the n-1 zeros of P_n' plus the two end points -1 and 1 (there n is the
polynomial degree; callers here pass the degree N explicitly).

Pins (tests/test_oracle_1d.py): nodes against numpy's Legendre-series roots,
symmetry, the quadrature weights summing to 2 and integrating x^m exactly for
m <= 2N-1 (textbook GLL exactness).
"""
from __future__ import annotations

import numpy as np


def legendre(N: int, x):
    """P_N(x), P_N'(x), P_N''(x) by the three-term recurrence.

    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1};
    P_{k+1}' = P_{k-1}' + (2k+1) P_k;   P_{k+1}'' = P_{k-1}'' + (2k+1) P_k'.
    """
    x = np.asarray(x, dtype=np.float64)
    p0, p1 = np.ones_like(x), x.copy()
    d0, d1 = np.zeros_like(x), np.ones_like(x)
    s0, s1 = np.zeros_like(x), np.zeros_like(x)
    if N == 0:
        return p0, d0, s0
    for k in range(1, N):
        p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        d2 = d0 + (2 * k + 1) * p1
        s2 = s0 + (2 * k + 1) * d1
        p0, p1, d0, d1, s0, s1 = p1, p2, d1, d2, s1, s2
    return p1, d1, s1


def legendre_table(N: int, x):
    """Matrices P[j,k] = P_k(x_j), P'[j,k], P''[j,k] for k = 0..N."""
    x = np.asarray(x, dtype=np.float64)
    P = np.zeros((x.size, N + 1))
    D = np.zeros_like(P)
    S = np.zeros_like(P)
    P[:, 0] = 1.0
    if N >= 1:
        P[:, 1] = x
        D[:, 1] = 1.0
    for k in range(1, N):
        P[:, k + 1] = ((2 * k + 1) * x * P[:, k] - k * P[:, k - 1]) / (k + 1)
        D[:, k + 1] = D[:, k - 1] + (2 * k + 1) * P[:, k]
        S[:, k + 1] = S[:, k - 1] + (2 * k + 1) * D[:, k]
    return P, D, S


def gll_nodes(N: int):
    """GLL nodes x_0=-1 < ... < x_N=1 and weights w_j = 2 / (N (N+1) P_N(x_j)^2).

    Interior nodes: Newton on P_N' from the Chebyshev-Gauss-Lobatto guesses
    -cos(pi j / N), with P_N'' taken from the recurrence.
    """
    if N < 2:
        raise ValueError("degree must be >= 2")
    x = -np.cos(np.pi * np.arange(N + 1) / N)
    xi = x[1:-1].copy()
    for _ in range(100):
        _, d1, d2 = legendre(N, xi)
        step = d1 / d2
        xi -= step
        if np.max(np.abs(step)) < 1e-16:
            break
    x[1:-1] = xi
    x[0], x[-1] = -1.0, 1.0
    pN, _, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * pN * pN)
    return x, w


def gauss_nodes(N: int):
    """The N zeros of P_N (Gauss-Legendre points), by Newton from -cos(pi (j+1/2)/N)."""
    g = -np.cos(np.pi * (np.arange(N) + 0.5) / N)
    for _ in range(100):
        p, d1, _ = legendre(N, g)
        step = p / d1
        g -= step
        if np.max(np.abs(step)) < 1e-16:
            break
    return g
