"""Non-zero Dirichlet data by lifting (oracle; test infrastructure).

The problem statement (eq. pblm:time:A-B) prescribes u = g on the boundary of
[-1, 1]^d.  With the unknowns at all GLL nodes, the equations are u = g at
every boundary node and the collocated PDE at the interior collocation grid,

    sum_k (R_1 (x) .. (x) L_k (x) .. (x) R_d) u_full = b(eta),

where R_k, L_k = beta_k D_k - eps D2_k are the full (n_k - 2) x n_k 1D matrices
of ``collocation.op1d`` (rows: collocation points; columns: every GLL node,
boundary nodes included).  Any grid function G that equals g on the boundary
lifts the data: u_full = G + w with w zero on the boundary, and the interior
values of w solve the zero-data system of ``operator`` (interior columns only)
with the source

    b_g = b - (c_mass M_full + c_op A_full) G,

after which u = w + G restricted to the interior nodes.  When G is a TT on the
full GLL grid, A_full G is a TT-matrix-by-TT product with the rectangular
cores

    first [L_1  R_1],  middle [[R_k, 0], [L_k, R_k]],  last [R_d; L_d],

the rank-2 pattern of ``operator.ttm_cores`` with every GLL node as a column,
so b_g is a TT too (TT lifting).  The interior values of G cancel: they enter
b_g through A_int and come back when G is added to w.

Pins (tests/test_oracle_dirichlet.py): a polynomial solution of degree
<= N in every variable with non-zero boundary values is reproduced to
rounding; the TT lifting equals its dense definition; the solution does not
depend on the interior values of G; zero data gives the zero-data solve; a
smooth non-polynomial solution converges spectrally.
"""
from __future__ import annotations

from functools import reduce

import numpy as np

from . import tt as T
from .operator import dense as dense_interior


def full_ttm_cores(ops, c_mass: float = 0.0, c_op: float = 1.0):
    """Rank-2 TT-matrix cores (R_{k-1}, n_k - 2, n_k, R_k) of
    c_mass M_full + c_op A_full: rows at the collocation points, columns at
    every GLL node."""
    d = len(ops)
    cores = []
    for k, o in enumerate(ops):
        R = o.R
        L = c_op * (o.beta * o.D - o.eps * o.D2)
        m, n = R.shape
        if d == 1:
            c = np.zeros((1, m, n, 1))
            c[0, :, :, 0] = L + c_mass * R
        elif k == 0:
            c = np.zeros((1, m, n, 2))
            c[0, :, :, 0] = L + c_mass * R
            c[0, :, :, 1] = R
        elif k == d - 1:
            c = np.zeros((2, m, n, 1))
            c[0, :, :, 0] = R
            c[1, :, :, 0] = L
        else:
            c = np.zeros((2, m, n, 2))
            c[0, :, :, 0] = R
            c[1, :, :, 0] = L
            c[1, :, :, 1] = R
        cores.append(c)
    return cores


def dense_full(ops, c_mass: float = 0.0, c_op: float = 1.0):
    """c_mass M_full + c_op A_full as a dense (prod (n_k - 2)) x (prod n_k) matrix."""
    d = len(ops)
    out = 0.0
    for k in range(d):
        mats = [o.R for o in ops]
        mats[k] = ops[k].beta * ops[k].D - ops[k].eps * ops[k].D2
        out = out + reduce(np.kron, mats)
    out = c_op * out
    if c_mass != 0.0:
        out = out + c_mass * reduce(np.kron, [o.R for o in ops])
    return out


def interior(G):
    """The interior slice of a TT on the full GLL grid."""
    return [c[:, 1:-1, :].copy() for c in G]


def lifted_source_tt(ops, b, G, c_mass: float = 0.0, c_op: float = 1.0):
    """b_g = b - (c_mass M_full + c_op A_full) G as a TT."""
    AG = T.matvec(full_ttm_cores(ops, c_mass, c_op), G)
    return T.add(b, T.scale(AG, -1.0))


def dense_solve(ops, b, G, c_mass: float = 0.0, c_op: float = 1.0):
    """Interior values of u from the full-grid system with u = G on the
    boundary nodes (direct solve; tiny grids).  Returns the interior array."""
    shape_full = [o.n for o in ops]
    g = T.full(G)
    inner = tuple(slice(1, -1) for _ in ops)
    mask = np.ones(shape_full, dtype=bool)
    mask[inner] = False
    gb = np.where(mask, g, 0.0).ravel()        # boundary values, zero inside
    rhs = T.full(b).ravel() - dense_full(ops, c_mass, c_op) @ gb
    u = np.linalg.solve(dense_interior(ops, c_mass, c_op), rhs)
    return u.reshape([o.n - 2 for o in ops])


def full_solution_tt(problem, ops):
    """u* (the problem's separable terms) sampled at every GLL node."""
    from .operator import separable_tt
    vecs = [[t.factors[k](ops[k].x) for k in range(problem.d)] for t in problem.terms]
    return separable_tt(vecs, [t.coef for t in problem.terms])
