"""Pins of the variable-coefficient oracle (eq. pblm:time:A with beta_k(x_k)
and a reaction rho0 + sum_k rho_k(x_k))."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import operator as O
from oracle import solve as S
from oracle import tt as T
from oracle import varcoef as V


def _vc(d, n, ratio=0.05, seed=3, prod=False):
    vp = W.config_varcoef(seed=seed, d=d, n=n, ratio=ratio)
    vc = V.VarCoef(np.asarray(vp.problem.beta), [vp.beta_fn(k) for k in range(d)],
                   [vp.rho_fn(k) for k in range(d)], vp.rho0,
                   [vp.prod_fn(k) for k in range(d)] if prod else None)
    vp.prod = prod
    return vp, vc


@pytest.mark.parametrize("prod", [False, True])
@pytest.mark.parametrize("d,n", [(1, 7), (2, 6), (3, 5)])
def test_operator_is_exact_on_polynomials(d, n, prod):
    vp, vc = _vc(d, n, prod=prod)
    p = vp.problem
    ops = V.build(p, vc)
    rng = np.random.default_rng(d)
    # u = prod_k (1 - x^2) q_k(x), degree n - 1 = N in each variable
    qs = [np.polynomial.Polynomial(rng.standard_normal(n - 2)) for _ in range(d)]
    w = np.polynomial.Polynomial([1.0, 0.0, -1.0])
    ps = [w * q for q in qs]
    u = T.full([ps[k](ops[k].x[1:-1]).reshape(1, -1, 1) for k in range(d)])
    Au = (V.dense(ops) @ u.ravel()).reshape(u.shape)
    # -eps Lap u + sum_k beta_k(x_k) d_k u + rho(x) u at the collocation grid
    grids = np.meshgrid(*[o.eta for o in ops], indexing="ij")
    val = [ps[k](grids[k]) for k in range(d)]
    want = np.zeros_like(Au)
    uval = np.prod(val, axis=0)
    rho = vp.rho0 + sum(vp.rho_fn(k)(grids[k]) for k in range(d))
    if prod:
        rho = rho + np.prod([vp.prod_fn(k)(grids[k]) for k in range(d)], axis=0)
    for k in range(d):
        others = np.prod([val[j] for j in range(d) if j != k], axis=0) if d > 1 else 1.0
        want += others * (vp.beta_fn(k)(grids[k]) * ps[k].deriv(1)(grids[k]) - p.eps * ps[k].deriv(2)(grids[k]))
    want += rho * uval
    assert np.allclose(Au, want, rtol=0, atol=1e-10 * np.abs(want).max())


def test_constant_coefficients_reduce_to_the_operator_module():
    p = W.config1(d=2, n=8, ratio=0.02)
    vc = V.VarCoef(np.asarray(p.beta), [None, None], [None, None], 0.0)
    ops_v = V.build(p, vc)
    ops_c = O.build(p)
    for a, b in zip(ops_v, ops_c):
        assert np.allclose(a.Lt, b.Lt, rtol=0, atol=1e-12 * np.abs(b.Lt).max())
        assert np.array_equal(a.Rt, b.Rt)


def test_source_is_the_pde_applied_to_the_solution():
    vp, vc = _vc(2, 8)
    p = vp.problem
    ops = V.build(p, vc)
    b = T.full(V.source_tt(p, ops))
    X, Y = np.meshgrid(ops[0].eta, ops[1].eta, indexing="ij")
    want = np.zeros_like(X)
    grids = (X, Y)
    for t in p.terms:
        f = [t.factors[k] for k in range(2)]
        u = t.coef * f[0](X) * f[1](Y)
        for k in range(2):
            o = 1 - k
            want += t.coef * f[o](grids[o]) * (vp.beta_fn(k)(grids[k]) * f[k](grids[k], 1)
                                               - p.eps * f[k](grids[k], 2))
        want += (vp.rho0 + vp.rho_fn(0)(X) + vp.rho_fn(1)(Y)) * u
    assert np.allclose(b, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_discrete_solution_converges_spectrally():
    errs = []
    for n in (8, 12, 16):
        vp, vc = _vc(2, n, ratio=0.05)
        p = vp.problem
        ops = V.build(p, vc)
        u = S.dense_solve(ops, V.source_tt(p, ops))
        want = T.full(O.solution_tt(p, ops))
        errs.append(np.abs(u - want).max() / np.abs(want).max())
    assert errs[1] < 0.2 * errs[0] and errs[2] < 0.2 * errs[1], errs


@pytest.mark.parametrize("d", [1, 2, 3])
def test_rank3_tt_matrix_is_the_dense_operator(d):
    vp, vc = _vc(d, 5, prod=True)
    ops = V.build(vp.problem, vc)
    for cm, co in ((0.0, 1.0), (1.5, 0.3)):
        assert np.allclose(T.ttm_full(V.ttm_cores(ops, cm, co)), V.dense(ops, cm, co), rtol=0, atol=1e-10)


def test_product_reaction_source_and_convergence():
    # the source is the PDE with the product reaction applied pointwise, and
    # the discrete solution converges spectrally
    vp, vc = _vc(2, 8, prod=True)
    p = vp.problem
    ops = V.build(p, vc)
    b = T.full(V.source_tt(p, ops))
    X, Y = np.meshgrid(ops[0].eta, ops[1].eta, indexing="ij")
    grids = (X, Y)
    want = np.zeros_like(X)
    rho = vp.rho0 + vp.rho_fn(0)(X) + vp.rho_fn(1)(Y) + vp.prod_fn(0)(X) * vp.prod_fn(1)(Y)
    for t in p.terms:
        f = [t.factors[k] for k in range(2)]
        u = t.coef * f[0](X) * f[1](Y)
        for k in range(2):
            o = 1 - k
            want += t.coef * f[o](grids[o]) * (vp.beta_fn(k)(grids[k]) * f[k](grids[k], 1)
                                               - p.eps * f[k](grids[k], 2))
        want += rho * u
    assert np.allclose(b, want, rtol=0, atol=1e-12 * np.abs(want).max())
    errs = []
    for n in (8, 12, 16):
        vp, vc = _vc(2, n, ratio=0.05, prod=True)
        ops = V.build(vp.problem, vc)
        u = np.linalg.solve(V.dense(ops), T.full(V.source_tt(vp.problem, ops)).ravel())
        want = T.full(O.solution_tt(vp.problem, ops)).ravel()
        errs.append(np.abs(u - want).max() / np.abs(want).max())
    assert errs[1] < 0.2 * errs[0] and errs[2] < 0.2 * errs[1], errs
