"""Unified space-time collocation (oracle; test infrastructure).

The paper solves the time-dependent problem (eq. pblm:time:A-C) either by
time stepping (Crank-Nicolson, backward Euler: ``solve.cn_step``,
``solve.be_step``) or in the unified space-time formulation, where time is one
more collocated dimension (Methods overview; Results, "Global Accuracy": the
time interval is mapped onto [-1, 1], the initial condition is a boundary
condition at t = -1, and at t = 1 the solution is whatever the scheme gives).
On [0, T] mapped to s in [-1, 1],

    (2/T) du/ds - eps Laplace u + beta . grad u = b,
    u(x, s = -1) = u0(x),   u = 0 on the spatial boundary.

Time is represented, like every dimension, by the Lagrange basis on the n_t
Gauss-Lobatto-Legendre nodes s_0 = -1 < ... < s_N = 1 (N = n_t - 1).  The
initial condition fixes the value at s_0, so the N time unknowns are s_1..s_N.
The time operator (2/T) d/ds is pure transport towards s = +1.  The
superconsistent points of a transport operator (eps -> 0 in Overview (ii))
are the zeros of P_N; with only the inflow end constrained there is no
outflow root to drop, so the N collocation times are the N Gauss points g_i.
This choice is a reading: the paper does not print the time nodes of its
space-time runs.

With the unknowns ordered time first, then x_1 .. x_d, the discrete operator is
the Kronecker sum over d + 1 dimensions,

    A_st = Lt_t (x) M_x  +  Rt_t (x) A_x,
    Rt_t[i, j] = l_j(g_i),  Lt_t[i, j] = (2/T) l_j'(g_i),   j = 1 .. N,

where M_x = Rt_1 (x) ... (x) Rt_d and A_x are the spatial mass matrix and
operator of ``operator``.  It is the same rank-2 TT-matrix as the steady one,
with the time dimension in front.  The initial condition enters through the
column j = 0 of the time matrices:

    b_st = b(g, eta) - Lt_t[:, 0] (x) (M_x u0) - Rt_t[:, 0] (x) (A_x u0).

Pins (tests/test_oracle_spacetime.py): the time matrices are exact on
polynomials of degree <= N and the collocation times are the zeros of P_N;
a space-time solution that is a polynomial of degree <= N in every variable
and vanishes on the spatial boundary is reproduced to rounding (this fixes the
lifting, its sign and the 2/T scaling); the TT-matrix and the lifted TT source
equal their dense Kronecker forms; the discrete solution of e^{s} times spatial
sines converges spectrally in n_t; AMEn on the space-time TT-matrix reaches the
dense solution.
"""
from __future__ import annotations

from dataclasses import dataclass, replace
from functools import reduce

import numpy as np

from workloads import SpaceTimeProblem  # noqa: F401  (parameters only)

from . import operator as O
from . import tt as T
from .collocation import lagrange_matrices
from .gll import gauss_nodes, gll_nodes


@dataclass
class TimeOp1D:
    """Time pieces, n GLL nodes, N = n - 1 unknowns (s_1 .. s_N) and N Gauss
    collocation times.  ``Rt``, ``Lt`` are N x N (unknown columns); ``r0``,
    ``l0`` the columns of the initial-condition node s_0 = -1."""
    n: int
    x: np.ndarray
    g: np.ndarray
    Rt: np.ndarray
    Lt: np.ndarray
    r0: np.ndarray
    l0: np.ndarray
    T: float


def time_op1d(n: int, T_len: float) -> TimeOp1D:
    """Time matrices for n GLL nodes on [0, T_len] mapped onto [-1, 1]."""
    N = n - 1
    x, _ = gll_nodes(N)
    g = gauss_nodes(N)
    R, D, _ = lagrange_matrices(x, g)
    scale = 2.0 / T_len
    return TimeOp1D(n, x, g, R[:, 1:].copy(), scale * D[:, 1:], R[:, 0].copy(), scale * D[:, 0], T_len)


def build(st: SpaceTimeProblem):
    """(time pieces, spatial 1D pieces)."""
    return time_op1d(st.n_t, st.T), O.build(st.space)


def dense(top: TimeOp1D, ops):
    """A_st as a dense matrix (tiny grids only)."""
    Mx = reduce(np.kron, [o.Rt for o in ops])
    Ax = O.dense(ops, 0.0, 1.0)
    return np.kron(top.Lt, Mx) + np.kron(top.Rt, Ax)


def ttm_cores(top: TimeOp1D, ops):
    """Rank-2 TT-matrix cores of A_st over the d + 1 dimensions, time first:
    the Kronecker sum of ``operator.ttm_cores`` with Lt_t, Rt_t in front."""
    return O.ttm_cores([top] + list(ops), 0.0, 1.0)


def solution_tt(st: SpaceTimeProblem, top: TimeOp1D, ops):
    """u* at the unknowns: time nodes s_1..s_N, interior spatial GLL nodes."""
    vecs = []
    for t, ft in zip(st.space.terms, st.time_factors):
        vecs.append([ft(top.x[1:])] + [t.factors[k](ops[k].x[1:-1]) for k in range(st.space.d)])
    return O.separable_tt(vecs, [t.coef for t in st.space.terms])


def initial_tt(st: SpaceTimeProblem, ops):
    """u0 = u*(x, s = -1) at the interior spatial GLL nodes (a d-dimensional TT)."""
    vecs, coefs = [], []
    for t, ft in zip(st.space.terms, st.time_factors):
        vecs.append([t.factors[k](ops[k].x[1:-1]) for k in range(st.space.d)])
        coefs.append(t.coef * float(ft(np.array([-1.0]))[0]))
    return O.separable_tt(vecs, coefs)


def source_tt(st: SpaceTimeProblem, top: TimeOp1D, ops):
    """b = (2/T) du*/ds - eps Laplace u* + beta . grad u* on the collocation
    grid (g, eta), before the initial-condition lifting: per separable term
    the time derivative term plus the spatial source times phi_t(g)."""
    total = None
    scale = 2.0 / st.T
    for t, ft in zip(st.space.terms, st.time_factors):
        one = replace(st.space, terms=[t])
        spatial = O.source_tt(one, ops)                      # (-eps Lap + beta.grad) of prod phi_k
        mass = O.separable_tt([[t.factors[k](ops[k].eta) for k in range(st.space.d)]], [t.coef])
        part = T.add(_prepend(ft(top.g), spatial), _prepend(scale * ft(top.g, 1), mass))
        total = part if total is None else T.add(total, part)
    return total


def lifted_source_tt(st: SpaceTimeProblem, top: TimeOp1D, ops):
    """b_st = b - Lt_t[:, 0] (x) (M_x u0) - Rt_t[:, 0] (x) (A_x u0)."""
    b = source_tt(st, top, ops)
    u0 = initial_tt(st, ops)
    Mu0 = T.matvec(O.ttm_cores(ops, 1.0, 0.0), u0)
    Au0 = T.matvec(O.ttm_cores(ops, 0.0, 1.0), u0)
    b = T.add(b, _prepend(-top.l0, Mu0))
    return T.add(b, _prepend(-top.r0, Au0))


def dense_solve(st: SpaceTimeProblem, top: TimeOp1D, ops):
    """Solve A_st u = b_st directly (tiny grids); returns the full array
    indexed (s_1..s_N, x_1, .., x_d)."""
    b = T.full(lifted_source_tt(st, top, ops))
    u = np.linalg.solve(dense(top, ops), b.ravel())
    return u.reshape(b.shape)


def _prepend(v, cores):
    """The TT of v (x) X for a vector v and a TT X (rank 1 between them)."""
    c0 = np.asarray(v, dtype=np.float64).reshape(1, -1, 1)
    return [c0] + [c.copy() for c in cores]
