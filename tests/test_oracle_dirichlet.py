"""Pins of the Dirichlet-data lifting oracle (eq. pblm:time:B: u = g on the
boundary; the data enter the interior equations through the boundary columns
of the full 1D matrices)."""
import numpy as np
import pytest

import workloads as W
from oracle import dirichlet as DI
from oracle import operator as O
from oracle import solve as S
from oracle import tt as T


def _problem(d, n, terms, ratio=0.05, seed=11):
    beta = W.random_unit_vector(d, np.random.default_rng(seed))
    return W.Problem(f"dir d={d} n={n}", d, (n,) * d, beta, ratio * W.EDGE_LENGTH, terms, tol=1e-12, rmax=20)


def _poly_terms(d):
    # degree 3 in every variable, non-zero at +-1
    f1 = W.Factor("poly", c=(1.0, 0.4, -0.3, 0.2))
    f2 = W.Factor("poly", c=(0.5, -1.0, 0.0, 0.7))
    return [W.Term(1.0, (f1,) * d), W.Term(-0.6, (f2,) * d)]


@pytest.mark.parametrize("d,n", [(1, 6), (2, 6), (3, 5)])
def test_polynomial_solution_with_boundary_values_is_reproduced(d, n):
    p = _problem(d, n, _poly_terms(d))
    ops = O.build(p)
    b = O.source_tt(p, ops)
    G = DI.full_solution_tt(p, ops)
    u = DI.dense_solve(ops, b, G)
    want = T.full(O.solution_tt(p, ops))
    assert np.abs(want).max() > 0.1
    assert np.linalg.norm(u - want) <= 1e-11 * np.linalg.norm(want)


def test_dropping_the_data_or_flipping_its_sign_fails():
    p = _problem(2, 6, _poly_terms(2))
    ops = O.build(p)
    b = O.source_tt(p, ops)
    G = DI.full_solution_tt(p, ops)
    want = T.full(O.solution_tt(p, ops))
    u0 = np.linalg.solve(O.dense(ops), T.full(b).ravel()).reshape(want.shape)
    assert np.linalg.norm(u0 - want) > 1e-2 * np.linalg.norm(want)
    bad = T.full(b).ravel() + DI.dense_full(ops) @ T.full(G).ravel()   # wrong sign of the lift
    u1 = np.linalg.solve(O.dense(ops), bad).reshape(want.shape)
    assert np.linalg.norm(u1 - want) > 1e-2 * np.linalg.norm(want)


def test_tt_lift_equals_its_dense_definition():
    p = _problem(3, 6, _poly_terms(3))
    ops = O.build(p)
    b = O.source_tt(p, ops)
    # any grid function on the full grid (not the solution, whose lift of its
    # own source vanishes)
    G = W.random_tt(3, 6, [1, 2, 3, 1], seed=9)
    for cm, co in ((0.0, 1.0), (1.0, 0.35)):
        got = T.full(DI.lifted_source_tt(ops, b, G, cm, co)).ravel()
        want = T.full(b).ravel() - DI.dense_full(ops, cm, co) @ T.full(G).ravel()
        assert np.allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
        # the full TT-matrix contracts to the dense Kronecker sum
        assert np.allclose(T.ttm_full(DI.full_ttm_cores(ops, cm, co)), DI.dense_full(ops, cm, co),
                           rtol=0, atol=1e-10)


def test_interior_values_of_the_lift_do_not_matter():
    p = _problem(2, 8, [W.Term(1.0, (W.Factor("exp", m=0.7), W.Factor("gauss", mu=0.2, s=0.5)))])
    ops = O.build(p)
    b = O.source_tt(p, ops)
    G = DI.full_solution_tt(p, ops)
    rng = np.random.default_rng(3)
    # add a random TT that vanishes on the boundary (zero first/last slices)
    H = W.random_tt(2, 8, [1, 3, 1], seed=4)
    for c in H:
        c[:, 0, :] = 0.0
        c[:, -1, :] = 0.0
    G2 = T.add(G, H)
    u1 = DI.dense_solve(ops, b, G)
    u2 = DI.dense_solve(ops, b, G2)
    assert np.linalg.norm(u1 - u2) <= 1e-12 * np.linalg.norm(u1)
    # and through the TT lift and AMEn: w + interior(G) is the same answer
    for GG in (G, G2):
        bg = DI.lifted_source_tt(ops, b, GG)
        w, res, _ = S.solve_collocation(ops, bg, [np.ones((1, 6, 1))] * 2, 1e-13, 20)
        u = T.full(T.add(w, DI.interior(GG)))
        assert np.linalg.norm(u - u1) <= 1e-10 * np.linalg.norm(u1)
    assert rng is not None


def test_zero_data_is_the_zero_data_solve():
    p = W.config0()
    ops = O.build(p)
    b = O.source_tt(p, ops)
    Z = [np.zeros((1, o.n, 1)) for o in ops]
    assert np.allclose(DI.dense_solve(ops, b, Z), S.dense_solve(ops, b), rtol=0, atol=1e-13)


def test_mass_term_lift_matches_dense():
    p = _problem(2, 7, [W.Term(1.0, (W.Factor("exp", m=-0.4), W.Factor("exp", m=0.9)))])
    ops = O.build(p)
    b = O.source_tt(p, ops)
    G = DI.full_solution_tt(p, ops)
    u = DI.dense_solve(ops, b, G, 2.0, 0.5)
    # the full-grid system, solved with the boundary rows u = g written out
    n = [o.n for o in ops]
    N = int(np.prod(n))
    Af = DI.dense_full(ops, 2.0, 0.5)
    rows = np.zeros((N, N))
    rhs = np.zeros(N)
    inner = np.zeros(n, dtype=bool)
    inner[1:-1, 1:-1] = True
    gi = T.full(G).ravel()
    rows[np.flatnonzero(inner)] = Af
    rhs[np.flatnonzero(inner)] = T.full(b).ravel()
    for i in np.flatnonzero(~inner.ravel()):
        rows[i, i] = 1.0
        rhs[i] = gi[i]
    uf = np.linalg.solve(rows, rhs).reshape(n)
    assert np.allclose(u, uf[1:-1, 1:-1], rtol=0, atol=1e-11 * np.abs(uf).max())


def test_smooth_data_converges_spectrally():
    errs = []
    for n in (6, 10, 14):
        p = W.config_dirichlet(d=2, n=n, ratio=0.05)
        ops = O.build(p)
        u = DI.dense_solve(ops, O.source_tt(p, ops), DI.full_solution_tt(p, ops))
        want = T.full(O.solution_tt(p, ops))
        errs.append(np.abs(u - want).max() / np.abs(want).max())
    assert errs[1] < 1e-2 * errs[0] and errs[2] < 1e-2 * errs[1] and errs[2] < 1e-8
