"""GPU parity: the alternating TT solve and the time steps against the oracle.

Parity rules: where the oracle has an exact dense solution (tiny grids) the
GPU solution must match it to 1e-10 relative (FP64 mode, tol 1e-12).  On
larger grids the hard check is the residual of the GPU's solution recomputed
by the oracle, which must be <= tol, plus the solution's distance to the
oracle's own AMEn solution, bounded by kappa-style 1e3 * tol (a derived bound).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import operator as O
from oracle import solve as OS
from oracle import tt as OT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2506_04732_gb300 as pkg
    torch.cuda.set_device(0)
    return pkg


def _setup(T, p):
    from paper_2506_04732_gb300 import problem as P
    op = P.build_operator(p)
    b = T.TT.from_cores(P.source_cores(p, op))
    m = [n - 2 for n in p.n]
    x = T.TT.from_cores([np.ones((1, mm, 1)) for mm in m], rcap=p.rmax + T.RANK_KICK)
    return op, b, x


def test_solve_config0_matches_dense_lu(T):
    p = W.config0()
    op, b, x = _setup(T, p)
    info = T.t2s2_solve(op, b, x, p.tol, p.rmax, p.max_sweeps)
    assert info.residual <= p.tol
    ops = O.build(p)
    ob = O.source_tt(p, ops)
    xd = OS.dense_solve(ops, ob)
    xg = OT.full(x.cores())
    assert np.linalg.norm(xg - xd) <= 1e-10 * np.linalg.norm(xd)
    # the oracle's own residual of the GPU solution
    assert OS.residual(O.ttm_cores(ops), ob, x.cores()) <= p.tol * 1.01
    # and the discrete solution is the spectrally accurate one
    us = OT.full(O.solution_tt(p, ops))
    assert np.linalg.norm(xg - us) <= 1e-11 * np.linalg.norm(us)


@pytest.mark.parametrize("plain", [False, True])
def test_solve_small_random_problem(T, plain):
    p = W.config1(d=3, n=10, ratio=0.01)
    p.plain_sc = plain
    op, b, x = _setup(T, p)
    info = T.t2s2_solve(op, b, x, 1e-11, 20, 30)
    ops = O.build(p)
    ob = O.source_tt(p, ops)
    xd = OS.dense_solve(ops, ob)
    assert info.residual <= 1e-11
    assert np.linalg.norm(OT.full(x.cores()) - xd) <= 1e-8 * np.linalg.norm(xd)


def test_solve_d5_residual_checked_by_oracle(T):
    p = W.config1(d=5, n=24, ratio=1e-2, rmax=16, tol=1e-8)
    op, b, x = _setup(T, p)
    info = T.t2s2_solve(op, b, x, p.tol, p.rmax, 30)
    ops = O.build(p)
    ob = O.source_tt(p, ops)
    r_or = OS.residual(O.ttm_cores(ops), ob, x.cores())
    assert info.residual <= p.tol
    assert abs(r_or - info.residual) <= 1e-3 * p.tol + 1e-6 * info.residual
    us = O.solution_tt(p, ops)
    assert OT.diff_norm(x.cores(), us) <= 1e-5 * OT.norm(us)


def test_solve_from_random_high_rank_guess(T):
    # a random rank-20 initial guess: the last core's local solves (right rank
    # 1) then see left ranks of 17 and more, beyond the 16-lane Gauss-Jordan
    # halves of the rank-1-right solver, while the first cores go through GMRES
    p = W.config1(d=4, n=24, ratio=1e-2, rmax=24, tol=1e-9)
    from paper_2506_04732_gb300 import problem as P
    op = P.build_operator(p)
    b = T.TT.from_cores(P.source_cores(p, op))
    m = [n - 2 for n in p.n]
    rng = np.random.default_rng(2506)
    r = [1, 20, 20, 20, 1]
    x0 = [rng.standard_normal((r[k], m[k], r[k + 1])) / np.sqrt(r[k] * m[k]) for k in range(p.d)]
    x = T.TT.from_cores(x0, rcap=p.rmax + T.RANK_KICK)
    info = T.t2s2_solve(op, b, x, p.tol, p.rmax, 30)
    assert info.status == 0 and info.residual <= p.tol
    ops = O.build(p)
    ob = O.source_tt(p, ops)
    r_or = OS.residual(O.ttm_cores(ops), ob, x.cores())
    assert r_or <= p.tol * 1.01
    assert abs(r_or - info.residual) <= 1e-3 * p.tol + 1e-6 * info.residual
    us = O.solution_tt(p, ops)
    assert OT.diff_norm(x.cores(), us) <= 1e-5 * OT.norm(us)


def test_solve_matches_oracle_amen(T):
    # two different iterates of the same solver family: both reach tol in the
    # oracle's residual, and they differ by at most a condition-style factor
    # (1e3, a derived bound) times tol
    p = W.sine_problem(d=4, n=14, ratio=1e-2, tol=1e-8, rmax=12)
    op, b, x = _setup(T, p)
    info = T.t2s2_solve(op, b, x, p.tol, p.rmax, 30)
    ops = O.build(p)
    ob = O.source_tt(p, ops)
    A = O.ttm_cores(ops)
    xo, ro, _ = OS.amen_solve(A, ob, [np.ones((1, 12, 1))] * 4, p.tol, p.rmax)
    assert info.residual <= p.tol and ro <= p.tol
    assert OS.residual(A, ob, x.cores()) <= p.tol * 1.01
    assert OT.diff_norm(x.cores(), xo) <= 1e3 * p.tol * OT.norm(xo)


def test_cn_step_matches_dense(T):
    p = W.config2(d=3, n=12, dt=0.01)
    from paper_2506_04732_gb300 import problem as P
    op = P.build_operator(p)
    ops = O.build(p)
    u0 = O.solution_tt(p, ops)
    u = T.TT.from_cores(P.solution_cores(p, op), rcap=16 + T.RANK_KICK)
    info = T.t2s2_cn_step(op, u, p.dt, 1e-12, 16)
    Mp = O.dense(ops, 1.0, 0.5 * p.dt)
    Mm = O.dense(ops, 1.0, -0.5 * p.dt)
    ud = np.linalg.solve(Mp, Mm @ OT.full(u0).ravel())
    assert info.residual <= 1e-12
    assert np.linalg.norm(OT.full(u.cores()).ravel() - ud) <= 1e-10 * np.linalg.norm(ud)


def test_be_step_matches_dense(T):
    p = W.config2(d=2, n=10, dt=0.05)
    from paper_2506_04732_gb300 import problem as P
    op = P.build_operator(p)
    ops = O.build(p)
    u0 = O.solution_tt(p, ops)
    u = T.TT.from_cores(P.solution_cores(p, op), rcap=10 + T.RANK_KICK)
    T.t2s2_be_step(op, u, p.dt, 1e-12, 10)
    ud = np.linalg.solve(O.dense(ops, 1.0, p.dt), O.dense(ops, 1.0, 0.0) @ OT.full(u0).ravel())
    assert np.linalg.norm(OT.full(u.cores()).ravel() - ud) <= 1e-10 * np.linalg.norm(ud)


def test_solve_config1_full_size(T):
    p = W.config1()
    op, b, x = _setup(T, p)
    import time
    torch.cuda.synchronize()
    t = time.time()
    info = T.t2s2_solve(op, b, x, p.tol, p.rmax, p.max_sweeps)
    torch.cuda.synchronize()
    print(f"config1 solve: {time.time() - t:.3f}s residual {info.residual:.2e} sweeps {info.sweeps} "
          f"rank {info.max_rank} local its {info.local_iters}")
    assert info.residual <= p.tol
    ops = O.build(p)
    r_or = OS.residual(O.ttm_cores(ops), O.source_tt(p, ops), x.cores())
    assert r_or <= p.tol * 1.01
    us = O.solution_tt(p, ops)
    assert OT.diff_norm(x.cores(), us) <= 1e-6 * OT.norm(us)


def test_solve_batched_matches_sequential(T):
    from paper_2506_04732_gb300 import problem as P
    probs = [W.config3(i) for i in range(6)]
    ops, bs, xs, xs_seq = [], [], [], []
    for p in probs:
        op = P.build_operator(p)
        ops.append(op)
        bs.append(T.TT.from_cores(P.source_cores(p, op)))
        m = [n - 2 for n in p.n]
        xs.append(T.TT.from_cores([np.ones((1, mm, 1)) for mm in m], rcap=p.rmax + T.RANK_KICK))
        xs_seq.append(T.TT.from_cores([np.ones((1, mm, 1)) for mm in m], rcap=p.rmax + T.RANK_KICK))
    infos = T.t2s2_solve_batched(ops, bs, xs, 1e-8, 16, 50, workers=3)
    for i, p in enumerate(probs):
        assert infos[i].status == 0 and infos[i].residual <= 1e-8
        seq = T.t2s2_solve(ops[i], bs[i], xs_seq[i], 1e-8, 16, 50)
        # the batched solve gives each instance a share of the SMs, which
        # changes the grid (and so the summation order) of its cooperative
        # kernels: the same iterates up to rounding, the same tolerance
        assert seq.residual <= 1e-8 and abs(seq.sweeps - infos[i].sweeps) <= 1
        assert T.t2s2_diff_norm(ops[i], xs[i], xs_seq[i]) <= 1e-6 * T.t2s2_norm(ops[i], xs_seq[i])
        ops_o = O.build(p)
        r = OS.residual(O.ttm_cores(ops_o), O.source_tt(p, ops_o), xs[i].cores())
        assert r <= 1.01e-8


def test_cn_step_config2_full_size_checked_by_oracle(T):
    # d=7, n=64 Gaussian pulse: the oracle recomputes the step equation
    # (M + dt/2 A) u1 = (M - dt/2 A) u0 on the GPU's u1; the bound is the rhs
    # rounding tolerance plus the solve tolerance.
    from paper_2506_04732_gb300 import problem as P
    p = W.config2()
    op = P.build_operator(p)
    u = T.TT.from_cores(P.solution_cores(p, op), rcap=p.rmax + T.RANK_KICK)
    info = T.t2s2_cn_step(op, u, p.dt, p.tol, p.rmax)
    assert info.residual <= p.tol and max(u.r) <= p.rmax + T.RANK_KICK
    ops = O.build(p)
    u0 = O.solution_tt(p, ops)
    lhs = OT.matvec(O.ttm_cores(ops, 1.0, 0.5 * p.dt), u.cores())
    rhs = OT.matvec(O.ttm_cores(ops, 1.0, -0.5 * p.dt), u0)
    assert OT.diff_norm(lhs, rhs) <= 2.0 * p.tol * OT.norm(rhs)
