"""Superconsistent collocation points and 1D Lagrange matrices (oracle; test infrastructure).

Overview (ii) of the paper: the equation is collocated on points that differ
from the representation points.  For the 1D model beta u' - eps u'' = 1
(eq. adv-diff-1d) they are the zeros of P_N' when diffusion dominates and the
zeros of P_N when convection dominates, with an intermediate set in between
that depends only on eps/|beta| and N (Fig. 1).  The paper does not print the
formula (its Methods section covers only the tensor-train part), so this module
follows a reading of Overview (ii):

    eta = roots in (-1, 1) of q(x) = eps P_N'(x) - beta P_N(x).

q is, up to the factor N(N+1), the 1D operator L = beta d/dx - eps d^2/dx^2
applied to the GLL nodal polynomial (1 - x^2) P_N'(x), because
((1 - x^2) P_N')' = -N (N+1) P_N.  Collocating at its zeros therefore makes the
discrete operator exact on polynomials of degree N+1, one degree more than the
basis: the scheme is consistent one degree beyond its trial space.  q has
degree N; when N roots fall inside (-1, 1) the one nearest the outflow end
x = sign(beta) is dropped (it leaves the interval through that end exactly when
eps = 2|beta| / (N(N+1))).  beta = 0, or the Plain-SC switch, gives the
interior GLL points (Overview (i)).

Pins (tests/test_oracle_1d.py): the two limits eps/|beta| -> infinity and
-> 0 stated in Overview (ii); dependence on eps/|beta| only; exactness of the
collocated operator on degree N+1 polynomials; mirror symmetry in beta;
polynomial exactness of R, D, D2 (degree <= N); and the qualitative claim of
Fig. 1 on eq. adv-diff-1d (bounded SC solution, oscillating Plain-SC one).  The
choice of this particular node family over Funaro's original rule is a reading
and is "parity unpinned" against the paper's own (unprinted) formula.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from numpy.polynomial import legendre as npleg

from .gll import gll_nodes, legendre, legendre_table


def sc_nodes(N: int, eps: float, beta: float, plain: bool = False):
    """The N-1 collocation points for degree N, per the reading above."""
    x, _ = gll_nodes(N)
    if plain or beta == 0.0:
        return x[1:-1].copy()
    # Legendre-series coefficients of q: P_N' = sum_{k = N-1, N-3, ...} (2k+1) P_k.
    c = np.zeros(N + 1)
    c[N] = -beta
    for k in range(N - 1, -1, -2):
        c[k] = eps * (2 * k + 1)
    roots = npleg.legroots(c)
    roots = np.real(roots[np.abs(np.imag(roots)) < 1e-8])
    roots = roots[np.isfinite(roots) & (np.abs(roots) < 1.5)]
    # Newton polish on q = eps P' - beta P, q' = eps P'' - beta P'.
    for _ in range(50):
        p, d1, d2 = legendre(N, roots)
        step = (eps * d1 - beta * p) / (eps * d2 - beta * d1)
        roots = roots - step
        if np.max(np.abs(step)) < 1e-16:
            break
    inside = np.sort(roots[(roots > -1.0) & (roots < 1.0)])
    if inside.size == N:
        inside = inside[:-1] if beta > 0 else inside[1:]
    if inside.size != N - 1:
        raise RuntimeError(f"superconsistent node count {inside.size} != {N - 1}")
    return inside


def lagrange_matrices(x, pts):
    """R[j,i] = l_i(pts_j), D[j,i] = l_i'(pts_j), D2[j,i] = l_i''(pts_j).

    l_i is the Lagrange polynomial of the representation points x (degree N).
    It is written in the Legendre basis, l_i = sum_k C[k,i] P_k with V C = I,
    V[m,k] = P_k(x_m), and differentiated term by term.
    """
    N = len(x) - 1
    V, _, _ = legendre_table(N, x)
    C = np.linalg.solve(V, np.eye(N + 1))
    P, P1, P2 = legendre_table(N, pts)
    return P @ C, P1 @ C, P2 @ C


@dataclass
class Op1D:
    """1D pieces for one dimension, n = N+1 GLL nodes, n' = n-2 interior unknowns.

    R, D, D2 are (n-2) x n (all representation points); Rt, Lt their interior
    columns, with Lt = beta D - eps D2 on the interior columns.
    """
    n: int
    x: np.ndarray
    w: np.ndarray
    eta: np.ndarray
    R: np.ndarray
    D: np.ndarray
    D2: np.ndarray
    Rt: np.ndarray
    Lt: np.ndarray
    beta: float
    eps: float


def op1d(n: int, eps: float, beta: float, plain: bool = False) -> Op1D:
    N = n - 1
    x, w = gll_nodes(N)
    eta = sc_nodes(N, eps, beta, plain)
    R, D, D2 = lagrange_matrices(x, eta)
    Rt, Dt, D2t = R[:, 1:-1], D[:, 1:-1], D2[:, 1:-1]
    return Op1D(n, x, w, eta, R, D, D2, Rt.copy(), beta * Dt - eps * D2t, beta, eps)
