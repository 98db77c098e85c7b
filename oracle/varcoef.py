"""Variable convection and reaction coefficients (oracle; test infrastructure).

Problem statement eq. pblm:time:A allows beta = beta(x) and a reaction
rho(x) f.  The paper's six-dimensional test takes each component of beta as a
function of its own coordinate only, beta_k = beta_k(x_k).  Collocated at the
point eta_j of the Cartesian grid, beta_k(eta_{j_k}) d_k u(eta_j) only scales
the rows of dimension k's 1D derivative, so the operator keeps the Kronecker
sum form with

    Lt_k = diag(beta_k(eta)) D_k - eps D2_k + diag(rho_k(eta)) Rt_k,

where the reaction is taken as a constant plus a sum of one-coordinate
functions, rho(x) = rho_0 + sum_k rho_k(x_k) (the constant is folded into the
first dimension).  Both keep the rank-2 TT-matrix of ``operator``.  A
reaction that is a product of one-coordinate functions (the paper's
six-dimensional test) adds a rank-1 Kronecker product instead, a rank-3
TT-matrix; it is not covered here.

The superconsistent points of dimension k depend on one convection speed;
with a variable beta_k they are chosen for a reference speed supplied with
the problem (a reading: the paper does not say which speed picks them).

Pins (tests/test_oracle_varcoef.py): the operator applied to grid values of a
tensor-product polynomial that vanishes on the boundary equals
-eps Laplace u + beta . grad u + rho u at the collocation grid exactly;
constant coefficients give ``operator``'s matrices; the manufactured source
is the PDE applied pointwise; the discrete solution converges spectrally.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np

from .collocation import Op1D, lagrange_matrices, sc_nodes
from .gll import gll_nodes


@dataclass
class VarCoef:
    """beta_k(x) per dimension (None: the constant beta_ref[k]), rho_k(x) per
    dimension (None: zero) and the constant rho0."""
    beta_ref: np.ndarray
    beta_fns: list
    rho_fns: list
    rho0: float = 0.0


def op1d_var(n: int, eps: float, beta_ref: float, beta_fn: Optional[Callable], rho_fn: Optional[Callable],
             rho_const: float, plain: bool = False) -> Op1D:
    """Op1D of one dimension with variable coefficients: R, D, D2 full
    (n - 2) x n, Rt and Lt their interior columns with the rows of D scaled by
    beta(eta) and the reaction added."""
    N = n - 1
    x, w = gll_nodes(N)
    eta = sc_nodes(N, eps, beta_ref, plain)
    R, D, D2 = lagrange_matrices(x, eta)
    b = beta_fn(eta) if beta_fn is not None else np.full(eta.shape, beta_ref)
    r = (rho_fn(eta) if rho_fn is not None else 0.0) + rho_const
    Lfull = b[:, None] * D - eps * D2 + (np.asarray(r) * np.ones_like(eta))[:, None] * R
    op = Op1D(n, x, w, eta, R, D, D2, R[:, 1:-1].copy(), Lfull[:, 1:-1].copy(), beta_ref, eps)
    op.Lfull = Lfull
    op.bvals = b
    op.rvals = np.asarray(r) * np.ones_like(eta)
    return op


def build(problem, vc: VarCoef):
    """Per-dimension pieces; rho0 goes to the first dimension."""
    return [op1d_var(problem.n[k], problem.eps, float(vc.beta_ref[k]), vc.beta_fns[k], vc.rho_fns[k],
                     vc.rho0 if k == 0 else 0.0, problem.plain_sc) for k in range(problem.d)]


def source_tt(problem, ops):
    """b = -eps Laplace u* + beta . grad u* + rho u* on the collocation grid
    for the separable terms of u*: per term and dimension k the factor
    beta_k(eta) phi_k' - eps phi_k'' + rho_k(eta) phi_k (rho0 with k = 0),
    a rank-2 TT per term."""
    total = None
    d = problem.d
    for t in problem.terms:
        cores = []
        for k in range(d):
            e = ops[k].eta
            f = t.factors[k]
            p = f(e)
            l = ops[k].bvals * f(e, 1) - problem.eps * f(e, 2) + ops[k].rvals * p
            m = len(e)
            if d == 1:
                c = np.zeros((1, m, 1)); c[0, :, 0] = l
            elif k == 0:
                c = np.zeros((1, m, 2)); c[0, :, 0] = l; c[0, :, 1] = p
            elif k == d - 1:
                c = np.zeros((2, m, 1)); c[0, :, 0] = p; c[1, :, 0] = l
            else:
                c = np.zeros((2, m, 2)); c[0, :, 0] = p; c[1, :, 0] = l; c[1, :, 1] = p
            cores.append(c)
        cores[0] = cores[0] * t.coef
        if total is None:
            total = cores
        else:
            from .tt import add
            total = add(total, cores)
    return total
