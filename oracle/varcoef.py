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
reaction that is a product of one-coordinate functions, prod_k pi_k(x_k) (the
paper's six-dimensional test), adds the Kronecker product
(x)_k diag(pi_k(eta)) Rt_k: a rank-3 TT-matrix,

    first [Lt_1  Rt_1  P_1],  middle [[Rt, 0, 0], [Lt, Rt, 0], [0, 0, P_k]],
    last [Rt; Lt; P_d],   P_k = diag(pi_k(eta)) Rt_k.

The superconsistent points of dimension k depend on one convection speed;
with a variable beta_k they are chosen for a reference speed supplied with
the problem (a reading: the paper does not say which speed picks them).

Pins (tests/test_oracle_varcoef.py): the operator applied to grid values of a
tensor-product polynomial that vanishes on the boundary equals
-eps Laplace u + beta . grad u + rho u at the collocation grid exactly (with
and without the product term); constant coefficients give ``operator``'s
matrices; the rank-3 TT-matrix contracts to the dense operator; the
manufactured source is the PDE applied pointwise; the discrete solution
converges spectrally.
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
    dimension (None: zero), the constant rho0 and the factors pi_k(x) of a
    product reaction prod_k pi_k(x_k) (None: no product term)."""
    beta_ref: np.ndarray
    beta_fns: list
    rho_fns: list
    rho0: float = 0.0
    prod_fns: Optional[list] = None


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
    """Per-dimension pieces; rho0 goes to the first dimension.  With a
    product reaction each piece also carries P = diag(pi_k(eta)) Rt."""
    ops = [op1d_var(problem.n[k], problem.eps, float(vc.beta_ref[k]), vc.beta_fns[k], vc.rho_fns[k],
                    vc.rho0 if k == 0 else 0.0, problem.plain_sc) for k in range(problem.d)]
    if vc.prod_fns is not None:
        for o, f in zip(ops, vc.prod_fns):
            o.pvals = np.asarray(f(o.eta), dtype=np.float64) * np.ones_like(o.eta)
            o.P = o.pvals[:, None] * o.Rt
    return ops


def dense(ops, c_mass: float = 0.0, c_op: float = 1.0):
    """c_mass M + c_op (A + the product reaction) as a dense matrix (tiny grids)."""
    from functools import reduce
    from .operator import dense as dense_sum
    out = dense_sum(ops, c_mass, c_op)
    if getattr(ops[0], "P", None) is not None:
        out = out + c_op * reduce(np.kron, [o.P for o in ops])
    return out


def ttm_cores(ops, c_mass: float = 0.0, c_op: float = 1.0):
    """TT-matrix cores of c_mass M + c_op (A + product reaction): the rank-2
    cores of ``operator`` without a product term, the rank-3 pattern above
    with one."""
    from .operator import ttm_cores as ttm2
    if getattr(ops[0], "P", None) is None:
        return ttm2(ops, c_mass, c_op)
    d = len(ops)
    cores = []
    for k, o in enumerate(ops):
        R, L, Pk = o.Rt, c_op * o.Lt, o.P
        m = R.shape[0]
        if d == 1:
            c = np.zeros((1, m, m, 1))
            c[0, :, :, 0] = L + c_mass * R + c_op * Pk
        elif k == 0:
            c = np.zeros((1, m, m, 3))
            c[0, :, :, 0] = L + c_mass * R
            c[0, :, :, 1] = R
            c[0, :, :, 2] = c_op * Pk
        elif k == d - 1:
            c = np.zeros((3, m, m, 1))
            c[0, :, :, 0] = R
            c[1, :, :, 0] = L
            c[2, :, :, 0] = Pk
        else:
            c = np.zeros((3, m, m, 3))
            c[0, :, :, 0] = R
            c[1, :, :, 0] = L
            c[1, :, :, 1] = R
            c[2, :, :, 2] = Pk
        cores.append(c)
    return cores


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
        if getattr(ops[0], "P", None) is not None:
            # the product reaction of this term: prod_k pi_k(eta) phi_k(eta), rank 1
            from .tt import add
            prod = [(ops[k].pvals * t.factors[k](ops[k].eta)).reshape(1, -1, 1) for k in range(d)]
            prod[0] = prod[0] * t.coef
            cores = add(cores, prod)
        if total is None:
            total = cores
        else:
            from .tt import add
            total = add(total, cores)
    return total
