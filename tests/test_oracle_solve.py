"""Pins for the oracle's solvers and time steps (dense algebra and closed forms)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import operator as O
from oracle import solve as S
from oracle import tt as T


def _ones(ops):
    return [np.ones((1, o.n - 2, 1)) for o in ops]


def test_amen_matches_dense_lu_config0():
    p = W.config0()
    ops = O.build(p)
    A, b = O.ttm_cores(ops), O.source_tt(p, ops)
    x, res, sweeps = S.amen_solve(A, b, _ones(ops), p.tol, p.rmax)
    xd = S.dense_solve(ops, b)
    assert res <= p.tol
    assert np.linalg.norm(T.full(x) - xd) <= 1e-10 * np.linalg.norm(xd)
    # the residual the solver reports agrees with dense algebra
    r = O.dense(ops) @ T.full(x).ravel() - T.full(b).ravel()
    assert abs(np.linalg.norm(r) / np.linalg.norm(T.full(b)) - res) < 1e-14


@pytest.mark.parametrize("plain", [False, True])
def test_amen_matches_dense_lu_random_problem(plain):
    rng = np.random.default_rng(7)
    p = W.config1(d=3, n=10, ratio=0.01)
    p.plain_sc = plain
    ops = O.build(p)
    A, b = O.ttm_cores(ops), O.source_tt(p, ops)
    x0 = [rng.standard_normal((1, 8, 1)) for _ in range(3)]
    x, res, _ = S.amen_solve(A, b, x0, 1e-11, 20)
    xd = S.dense_solve(ops, b)
    assert res <= 1e-11
    assert np.linalg.norm(T.full(x) - xd) <= 1e-8 * np.linalg.norm(xd)


def test_amen_uses_gmres_path_for_large_local_systems():
    p = W.config1(d=3, n=12, ratio=0.05)
    ops = O.build(p)
    A, b = O.ttm_cores(ops), O.source_tt(p, ops)
    # dense_max=0 forces the iterative local solver everywhere
    x, res, _ = S.amen_solve(A, b, _ones(ops), 1e-9, 12, dense_max=0)
    xd = S.dense_solve(ops, b)
    assert res <= 1e-9
    assert np.linalg.norm(T.full(x) - xd) <= 1e-6 * np.linalg.norm(xd)


@pytest.mark.parametrize("plain", [False, True])
def test_node_form_matches_dense_lu(plain):
    # AMEn in the node-to-node form M^-1 A reaches the dense LU solution of the
    # original collocation system, and reports that system's residual
    p = W.config1(d=3, n=10, ratio=0.01)
    p.plain_sc = plain
    ops = O.build(p)
    b = O.source_tt(p, ops)
    x, res, _ = S.solve_collocation(ops, b, _ones(ops), 1e-11, 20)
    xd = S.dense_solve(ops, b)
    assert res <= 1e-11
    assert np.linalg.norm(T.full(x) - xd) <= 1e-8 * np.linalg.norm(xd)
    r = O.dense(ops) @ T.full(x).ravel() - T.full(b).ravel()
    assert abs(np.linalg.norm(r) / np.linalg.norm(T.full(b)) - res) < 1e-13


def test_node_form_with_mass_term_matches_dense():
    p = W.config0()
    ops = O.build(p)
    b = O.source_tt(p, ops)
    x, res, _ = S.solve_collocation(ops, b, _ones(ops), 1e-12, 16, c_mass=2.5, c_op=0.3)
    xd = S.dense_solve(ops, b, 2.5, 0.3)
    assert res <= 1e-12
    assert np.linalg.norm(T.full(x) - xd) <= 1e-10 * np.linalg.norm(xd)


def test_node_form_operator_is_the_kronecker_sum_of_b():
    # M^-1 A = sum_k I (x) B_k (x) I with B_k = Rt_k^-1 Lt_k, densely
    p = W.config1(d=3, n=6, ratio=0.02)
    ops = O.build(p)
    nops = [S._NodeOp(o) for o in ops]
    M = O.dense(ops, 1.0, 0.0)
    want = np.linalg.solve(M, O.dense(ops, 0.0, 1.0))
    assert np.allclose(T.ttm_full(O.ttm_cores(nops)), want, rtol=0, atol=1e-10 * np.max(np.abs(want)))


def test_headline_problem_completes_in_the_node_form():
    # d = 6, n = 32 (the headline workload): one or two sweeps reach 1e-8 in the
    # residual of the original collocation system, at ranks <= rmax + kick
    p = W.config1()
    ops = O.build(p)
    b = O.source_tt(p, ops)
    x, res, sweeps = S.solve_collocation(ops, b, _ones(ops), p.tol, p.rmax, max_sweeps=2)
    assert res <= p.tol and sweeps <= 2
    assert max(T.ranks(x)) <= p.rmax + 8
    # the discrete solution is the spectrally accurate one
    us = O.solution_tt(p, ops)
    assert T.diff_norm(x, us) <= 1e-6 * T.norm(us)


def test_cn_step_matches_dense():
    p = W.config2(d=2, n=10, dt=0.02)
    ops = O.build(p)
    u0 = O.solution_tt(p, ops)
    u1, res, _ = S.cn_step(ops, u0, p.dt, 1e-12, 10)
    Mp = O.dense(ops, 1.0, 0.5 * p.dt)
    Mm = O.dense(ops, 1.0, -0.5 * p.dt)
    ud = np.linalg.solve(Mp, Mm @ T.full(u0).ravel())
    assert np.linalg.norm(T.full(u1).ravel() - ud) <= 1e-10 * np.linalg.norm(ud)


def test_be_step_matches_dense():
    p = W.config2(d=2, n=9, dt=0.05)
    ops = O.build(p)
    u0 = O.solution_tt(p, ops)
    u1, _, _ = S.be_step(ops, u0, p.dt, 1e-12, 10)
    ud = np.linalg.solve(O.dense(ops, 1.0, p.dt), O.dense(ops, 1.0, 0.0) @ T.full(u0).ravel())
    assert np.linalg.norm(T.full(u1).ravel() - ud) <= 1e-10 * np.linalg.norm(ud)


def test_cn_amplification_factor_closed_form_1d():
    # d = 1, beta = 0, Plain-SC: Rt = I and A = -eps D2, so each eigenmode
    # (lam, v) of A is scaled by (1 - dt lam / 2) / (1 + dt lam / 2) per step.
    n, eps, dt = 14, 0.3, 0.05
    p = W.Problem("heat1d", 1, (n,), np.zeros(1), eps, [], 1e-13, 4, plain_sc=True)
    ops = O.build(p)
    lam, V = np.linalg.eig(ops[0].Lt)
    assert np.max(np.abs(lam.imag)) < 1e-8 and np.min(lam.real) > 0
    lam, V = lam.real, V.real
    for j in (0, 3, n - 3):
        u0 = [V[:, j].reshape(1, n - 2, 1)]
        u1, _, _ = S.cn_step(ops, u0, dt, 1e-13, 4)
        g = (1 - dt * lam[j] / 2) / (1 + dt * lam[j] / 2)
        assert np.allclose(u1[0].ravel(), g * V[:, j], atol=1e-11)
