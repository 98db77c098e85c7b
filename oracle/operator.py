"""The d-dimensional collocation operator (oracle; test infrastructure).

Overview (ii)-(iii) and Fig. 3: superconsistency is applied dimension by
dimension, so the collocation grid is Cartesian, eta_j = (eta_{j_1}, ..., eta_{j_d}),
and the discrete operator of -eps Laplace + beta . grad on that grid is a sum of
Kronecker products of 1D matrices.  With zero Dirichlet data (eq. pblm:time:B
with g = 0) the unknowns are the values at the interior GLL points and

    A = sum_k  Rt_1 (x) ... (x) Lt_k (x) ... (x) Rt_d,     Lt_k = beta_k D_k - eps D2_k,

where Rt_k interpolates from the interior representation points to the
collocation points (the other dimensions are evaluated there, not at their
representation points).  The same operator is the rank-2 TT-matrix
(eq. tt-matrix-format) with cores

    first [Lt_1  Rt_1],  middle [[Rt_k, 0], [Lt_k, Rt_k]],  last [Rt_d; Lt_d].

The collocated time derivative gives the mass matrix M = Rt_1 (x) ... (x) Rt_d.

Pins (tests/test_oracle_operator.py): the dense operator applied to grid values
of a tensor-product polynomial that vanishes on the boundary equals
(-eps Laplace u + beta . grad u) at the collocation grid exactly; the TT-matrix
cores contract to the dense Kronecker sum; the manufactured-solution discrete
solve converges spectrally to u* (Results, "Global Accuracy").
"""
from __future__ import annotations

from functools import reduce

import numpy as np

from .collocation import Op1D, op1d


def build(problem):
    """Per-dimension 1D pieces for a workloads.Problem."""
    return [op1d(problem.n[k], problem.eps, float(problem.beta[k]), problem.plain_sc)
            for k in range(problem.d)]


def dense(ops, c_mass: float = 0.0, c_op: float = 1.0):
    """c_mass * M + c_op * A as a dense matrix (tiny grids only)."""
    d = len(ops)
    out = 0.0
    for k in range(d):
        mats = [o.Rt for o in ops]
        mats[k] = ops[k].Lt
        out = out + reduce(np.kron, mats)
    out = c_op * out
    if c_mass != 0.0:
        out = out + c_mass * reduce(np.kron, [o.Rt for o in ops])
    return out


def ttm_cores(ops, c_mass: float = 0.0, c_op: float = 1.0):
    """Rank-2 TT-matrix cores (R_{k-1}, n', n', R_k) of c_mass M + c_op A."""
    d = len(ops)
    cores = []
    for k, o in enumerate(ops):
        R, L = o.Rt, c_op * o.Lt
        m = R.shape[0]
        if d == 1:
            c = np.zeros((1, m, m, 1))
            c[0, :, :, 0] = L + c_mass * R
        elif k == 0:
            c = np.zeros((1, m, m, 2))
            c[0, :, :, 0] = L + c_mass * R
            c[0, :, :, 1] = R
        elif k == d - 1:
            c = np.zeros((2, m, m, 1))
            c[0, :, :, 0] = R
            c[1, :, :, 0] = L
        else:
            c = np.zeros((2, m, m, 2))
            c[0, :, :, 0] = R
            c[1, :, :, 0] = L
            c[1, :, :, 1] = R
        cores.append(c)
    return cores


def separable_tt(vectors_per_term, coefs):
    """TT of sum_t coefs[t] * (v_{t,1} (x) ... (x) v_{t,d}), rank = number of terms."""
    T = len(coefs)
    d = len(vectors_per_term[0])
    cores = []
    for k in range(d):
        n = len(vectors_per_term[0][k])
        if d == 1:
            c = np.zeros((1, n, 1))
            for t in range(T):
                c[0, :, 0] += coefs[t] * vectors_per_term[t][k]
        elif k == 0:
            c = np.zeros((1, n, T))
            for t in range(T):
                c[0, :, t] = coefs[t] * vectors_per_term[t][k]
        elif k == d - 1:
            c = np.zeros((T, n, 1))
            for t in range(T):
                c[t, :, 0] = vectors_per_term[t][k]
        else:
            c = np.zeros((T, n, T))
            for t in range(T):
                c[t, :, t] = vectors_per_term[t][k]
        cores.append(c)
    return cores


def solution_tt(problem, ops):
    """u* (the problem's separable terms) sampled at the interior GLL points."""
    vecs = [[t.factors[k](ops[k].x[1:-1]) for k in range(problem.d)] for t in problem.terms]
    return separable_tt(vecs, [t.coef for t in problem.terms])


def source_tt(problem, ops):
    """b = -eps Laplace u* + beta . grad u* sampled on the collocation grid.

    For one separable term prod_k phi_k: b = sum_k (prod_{m != k} phi_m(eta_m))
    * (beta_k phi_k' - eps phi_k'')(eta_k), a rank-2 TT built exactly (the paper
    derives sources from analytic solutions, Results "Global Accuracy").
    Each separable term contributes a rank-2 block; ranks add over terms.
    """
    d, eps = problem.d, problem.eps
    total = None
    for t in problem.terms:
        cores = []
        for k in range(d):
            e = ops[k].eta
            f = t.factors[k]
            p = f(e)
            l = float(problem.beta[k]) * f(e, 1) - eps * f(e, 2)
            n = len(e)
            if d == 1:
                c = np.zeros((1, n, 1)); c[0, :, 0] = l
            elif k == 0:
                c = np.zeros((1, n, 2)); c[0, :, 0] = l; c[0, :, 1] = p
            elif k == d - 1:
                c = np.zeros((2, n, 1)); c[0, :, 0] = p; c[1, :, 0] = l
            else:
                c = np.zeros((2, n, 2)); c[0, :, 0] = p; c[1, :, 0] = l; c[1, :, 1] = p
            cores.append(c)
        cores[0] = cores[0] * t.coef
        if total is None:
            total = cores
        else:
            from .tt import add
            total = add(total, cores)
    return total
