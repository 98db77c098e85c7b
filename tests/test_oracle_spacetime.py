"""Pins of the space-time oracle (time as one more collocated dimension;
Methods overview and Results "Global Accuracy")."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import workloads as W
from oracle import operator as O
from oracle import solve as S
from oracle import spacetime as ST
from oracle import tt as T


def _space(d, n, ratio, terms, seed=7):
    beta = W.random_unit_vector(d, np.random.default_rng(seed))
    return W.Problem(f"st d={d} n={n}", d, (n,) * d, beta, ratio * W.EDGE_LENGTH, terms,
                     tol=1e-10, rmax=20)


@pytest.mark.parametrize("n", [3, 6, 11])
def test_time_matrices_are_exact_on_polynomials(n):
    top = ST.time_op1d(n, 2.5)
    N = n - 1
    # the collocation times are the N zeros of P_N
    e = np.zeros(N + 1)
    e[N] = 1.0
    assert np.max(np.abs(npleg.legval(top.g, e))) < 1e-13
    rng = np.random.default_rng(n)
    for deg in range(N + 1):
        c = rng.standard_normal(deg + 1)
        p = np.polynomial.polynomial.polyval(top.x, c)
        want = np.polynomial.polynomial.polyval(top.g, c)
        dwant = (2.0 / 2.5) * np.polynomial.polynomial.polyval(top.g, np.polynomial.polynomial.polyder(c))
        assert np.allclose(top.r0 * p[0] + top.Rt @ p[1:], want, rtol=0, atol=1e-12)
        assert np.allclose(top.l0 * p[0] + top.Lt @ p[1:], dwant, rtol=0, atol=1e-11 * max(1, N * N))


def _poly_problem(d, n, n_t):
    # u* = (1 + s + s^2/2 + s^3/7) * prod_k (1 - x_k^2)(1 + x_k/3), degree 3 in s and 3 in x:
    # inside the discrete space when n_t >= 4 and n >= 4
    fx = W.Factor("poly", c=(1.0, 1.0 / 3.0, -1.0, -1.0 / 3.0))
    ft = W.Factor("poly", c=(1.0, 1.0, 0.5, 1.0 / 7.0))
    sp = _space(d, n, 0.05, [W.Term(1.3, (fx,) * d)])
    return ST.SpaceTimeProblem(sp, (ft,), n_t, 1.7)


@pytest.mark.parametrize("d", [1, 2])
def test_polynomial_space_time_solution_is_reproduced(d):
    st = _poly_problem(d, 6, 5)
    top, ops = ST.build(st)
    u = ST.dense_solve(st, top, ops)
    want = T.full(ST.solution_tt(st, top, ops))
    assert np.linalg.norm(u - want) <= 1e-11 * np.linalg.norm(want)


def test_lifting_sign_and_time_scale_matter():
    # the same check with the initial condition dropped, or with T wrong,
    # must fail: the polynomial solution has u0 != 0 and du/ds != 0
    st = _poly_problem(2, 6, 5)
    top, ops = ST.build(st)
    want = T.full(ST.solution_tt(st, top, ops))
    b = T.full(ST.source_tt(st, top, ops))
    u_nolift = np.linalg.solve(ST.dense(top, ops), b.ravel()).reshape(b.shape)
    assert np.linalg.norm(u_nolift - want) > 1e-3 * np.linalg.norm(want)
    st2 = ST.SpaceTimeProblem(st.space, st.time_factors, st.n_t, 2.0 * st.T)
    top2, _ = ST.build(st2)
    b2 = T.full(ST.lifted_source_tt(st, top, ops))
    u_wrongT = np.linalg.solve(ST.dense(top2, ops), b2.ravel()).reshape(b2.shape)
    assert np.linalg.norm(u_wrongT - want) > 1e-3 * np.linalg.norm(want)


def test_tt_matrix_and_lifted_source_match_dense_forms():
    st = _poly_problem(2, 5, 4)
    top, ops = ST.build(st)
    assert np.allclose(T.ttm_full(ST.ttm_cores(top, ops)), ST.dense(top, ops), rtol=0, atol=1e-11)
    # lifted source against its dense definition
    b = T.full(ST.source_tt(st, top, ops)).ravel()
    u0 = T.full(ST.initial_tt(st, ops)).ravel()
    Mx = O.dense(ops, 1.0, 0.0)
    Ax = O.dense(ops, 0.0, 1.0)
    want = b - np.kron(top.l0, Mx @ u0) - np.kron(top.r0, Ax @ u0)
    got = T.full(ST.lifted_source_tt(st, top, ops)).ravel()
    assert np.allclose(got, want, rtol=0, atol=1e-11 * np.linalg.norm(want))


def test_source_is_the_pde_applied_to_the_solution():
    # b at the collocation grid against finite formulas of u* = e^{s} prod sin(pi(x+1)/2)
    fx = W.Factor("sine", m=1)
    ft = W.Factor("exp", m=1.0)
    sp = _space(2, 6, 0.1, [W.Term(1.0, (fx, fx))])
    st = ST.SpaceTimeProblem(sp, (ft,), 5, 3.0)
    top, ops = ST.build(st)
    b = T.full(ST.source_tt(st, top, ops))
    g, e0, e1 = top.g, ops[0].eta, ops[1].eta
    S_, X, Y = np.meshgrid(g, e0, e1, indexing="ij")
    k = math.pi / 2
    u = np.exp(S_) * np.sin(k * (X + 1)) * np.sin(k * (Y + 1))
    ux = np.exp(S_) * k * np.cos(k * (X + 1)) * np.sin(k * (Y + 1))
    uy = np.exp(S_) * np.sin(k * (X + 1)) * k * np.cos(k * (Y + 1))
    lap = -2 * k * k * u
    want = (2.0 / 3.0) * u + sp.beta[0] * ux + sp.beta[1] * uy - sp.eps * lap
    assert np.allclose(b, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))


def test_exponential_in_time_converges_spectrally():
    fx = W.Factor("sine", m=1)
    ft = W.Factor("exp", m=1.0)
    sp = _space(1, 10, 0.1, [W.Term(1.0, (fx,))])
    errs = []
    for n_t in (3, 5, 7, 9):
        st = ST.SpaceTimeProblem(sp, (ft,), n_t, 2.0)
        top, ops = ST.build(st)
        u = ST.dense_solve(st, top, ops)
        want = T.full(ST.solution_tt(st, top, ops))
        errs.append(np.max(np.abs(u - want)) / np.max(np.abs(want)))
    # the error falls by orders of magnitude with every two time nodes, until
    # the spatial resolution (n = 10) floor
    assert errs[1] < 1e-2 * errs[0] and errs[2] < 1e-2 * errs[1]
    assert errs[3] < 1e-6


def test_amen_on_the_space_time_operator_reaches_the_dense_solution():
    fx = W.Factor("sine", m=1)
    fx2 = W.Factor("sine", m=2)
    ft = W.Factor("exp", m=0.7)
    sp = _space(2, 7, 0.05, [W.Term(1.0, (fx, fx)), W.Term(0.4, (fx2, fx))])
    st = ST.SpaceTimeProblem(sp, (ft, W.Factor("poly", c=(1.0, -0.5))), 6, 1.0)
    top, ops = ST.build(st)
    A = ST.ttm_cores(top, ops)
    b = ST.lifted_source_tt(st, top, ops)
    x0 = [np.ones((1, c.shape[1], 1)) for c in b]
    x, res, _ = S.amen_solve(A, b, x0, 1e-12, 20)
    assert res <= 1e-12
    ud = ST.dense_solve(st, top, ops)
    assert np.linalg.norm(T.full(x) - ud) <= 1e-10 * np.linalg.norm(ud)


def test_node_form_amen_on_the_space_time_operator_reaches_the_dense_solution():
    fx = W.Factor("sine", m=1)
    sp = _space(2, 7, 0.01, [W.Term(1.0, (fx, W.Factor("sine", m=2)))])
    st = ST.SpaceTimeProblem(sp, (W.Factor("exp", m=-0.5),), 6, 2.0)
    top, ops = ST.build(st)
    b = ST.lifted_source_tt(st, top, ops)
    x0 = [np.ones((1, c.shape[1], 1)) for c in b]
    x, res, _ = S.solve_collocation([top] + list(ops), b, x0, 1e-12, 20)
    assert res <= 1e-12
    ud = ST.dense_solve(st, top, ops)
    assert np.linalg.norm(T.full(x) - ud) <= 1e-10 * np.linalg.norm(ud)


def test_spacetime_workload_is_seeded_and_resolved():
    a, b = W.config_spacetime(), W.config_spacetime()
    assert np.array_equal(a.space.beta, b.space.beta) and a.space.terms == b.space.terms
    assert not np.array_equal(W.config_spacetime(seed=7).space.beta, a.space.beta)
    # a reduced instance of the same recipe: the discrete space-time solution
    # approaches the manufactured one as the grids grow (spectral accuracy)
    errs = []
    for n, n_t in ((8, 6), (16, 12)):
        st = W.config_spacetime(d=2, n=n, n_t=n_t, ratio=0.05)
        top, ops = ST.build(st)
        u = ST.dense_solve(st, top, ops)
        want = T.full(ST.solution_tt(st, top, ops))
        errs.append(np.max(np.abs(u - want)) / np.max(np.abs(want)))
    assert errs[1] < 1e-5 * errs[0] and errs[1] < 1e-7
