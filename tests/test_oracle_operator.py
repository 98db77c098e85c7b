"""Pins for the oracle's d-dimensional operator, sources and dense solve.

The operator is checked against exact calculus on tensor-product polynomials,
the TT-matrix cores against the dense Kronecker sum, and the discrete solution
against the manufactured solution (spectral accuracy, Results section).
"""
import itertools

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import workloads as W
from oracle import operator as O
from oracle import tt as T


def _poly_factor(rng, N):
    """(1 - x^2) q(x), deg q = N-2, as a Legendre series (value, d/dx, d2/dx2 callables)."""
    q = rng.standard_normal(N - 1)
    w = npleg.poly2leg([1.0, 0.0, -1.0])
    c = npleg.legmul(w, q)
    return [lambda x, c=c, k=k: npleg.legval(x, npleg.legder(c, k) if k else c) for k in range(3)]


@pytest.mark.parametrize("d,n", [(1, 9), (2, 7), (2, 12), (3, 6), (3, 9)])
def test_dense_operator_exact_on_polynomials(d, n):
    rng = np.random.default_rng(10 * d + n)
    N = n - 1
    beta = rng.standard_normal(d)
    p = W.Problem("t", d, (n,) * d, beta, 0.037, [], 1e-8, 8)
    ops = O.build(p)
    facs = [_poly_factor(rng, N) for _ in range(d)]
    # grid values at interior GLL points
    vals = [f[0](o.x[1:-1]) for f, o in zip(facs, ops)]
    u = vals[0]
    for v in vals[1:]:
        u = np.multiply.outer(u, v)
    Au = O.dense(ops) @ u.ravel()
    # exact -eps Laplace u + beta . grad u at the collocation grid
    ev = [[f[k](o.eta) for k in range(3)] for f, o in zip(facs, ops)]
    exact = 0.0
    for k in range(d):
        parts = [ev[m][0] for m in range(d)]
        parts[k] = beta[k] * ev[k][1] - p.eps * ev[k][2]
        t = parts[0]
        for v in parts[1:]:
            t = np.multiply.outer(t, v)
        exact = exact + t
    exact = np.asarray(exact).ravel()
    assert np.max(np.abs(Au - exact)) < 1e-11 * np.max(np.abs(exact)) * n ** 2


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_ttm_cores_contract_to_dense(d):
    rng = np.random.default_rng(d)
    p = W.Problem("t", d, tuple(int(v) for v in rng.integers(4, 7, d)), rng.standard_normal(d),
                  0.05, [], 1e-8, 8)
    ops = O.build(p)
    for cm, co in [(0.0, 1.0), (1.0, 0.25), (1.0, -0.25)]:
        assert np.allclose(T.ttm_full(O.ttm_cores(ops, cm, co)), O.dense(ops, cm, co),
                           atol=1e-12 * np.abs(O.dense(ops, cm, co)).max())


def test_source_tt_matches_pointwise():
    p = W.config1(d=3, n=7)
    ops = O.build(p)
    b = T.full(O.source_tt(p, ops))
    for idx in itertools.product(*[range(5)] * 3):
        pt = [ops[k].eta[idx[k]] for k in range(3)]
        val = 0.0
        for t in p.terms:
            f = [t.factors[k] for k in range(3)]
            for k in range(3):
                prod = t.coef
                for m in range(3):
                    if m == k:
                        prod *= p.beta[k] * f[k](pt[k], 1) - p.eps * f[k](pt[k], 2)
                    else:
                        prod *= f[m](pt[m])
                val += prod
        assert abs(b[idx] - val) < 1e-12 * max(1.0, abs(val))


def test_config0_dense_solution_is_spectrally_accurate():
    # Results, "Global Accuracy": exponential decay of the error for a smooth
    # manufactured solution.  u* = prod sin(pi (x+1)/2).
    errs = []
    for n in (6, 8, 10, 12, 14, 16):
        p = W.config0()
        p.n = (n,) * 3
        ops = O.build(p)
        u = np.linalg.solve(O.dense(ops), T.full(O.source_tt(p, ops)).ravel())
        us = T.full(O.solution_tt(p, ops)).ravel()
        errs.append(np.linalg.norm(u - us) / np.linalg.norm(us))
    assert errs[-1] < 1e-12
    for a, b in zip(errs[:-2], errs[1:-1]):
        assert b < a / 3.0      # at least geometric decay per two degrees
    # TT rank of the separable u* is one (separable data, Methods)
    p = W.config0()
    ops = O.build(p)
    assert T.ranks(O.solution_tt(p, ops)) == [1, 1, 1, 1]


def test_plain_switch_gives_identity_interpolation():
    p = W.config0()
    p.plain_sc = True
    for o in O.build(p):
        assert np.allclose(o.Rt, np.eye(o.n - 2), atol=1e-13)
