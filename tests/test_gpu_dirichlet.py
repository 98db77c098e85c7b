"""GPU parity of non-zero Dirichlet data (row N4, eq. pblm:time:B) against the
lifting oracle (oracle/dirichlet.py).

The data g are passed as a TT on the full GLL grid.  The tests use g = u* +
H with H zero on the boundary but not inside, so that the lifted source is
far from zero and the interior values of g must cancel (they do not change
the solution).

* the lifted source b - (c_mass M_full + c_op A_full) g against the oracle's;
* the solve against the oracle's dense full-grid solve to 1e-10 (FP64), and
  against the polynomial u* it reproduces;
* zero data (None) is the plain solve;
* at d = 5, n = 24 (the Dirichlet workload): the oracle recomputes the
  residual of the interior equations, and the solution lies within 1e-6 of u*.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import dirichlet as DI
from oracle import operator as O
from oracle import tt as OT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2506_04732_gb300 as pkg
    torch.cuda.set_device(0)
    return pkg


def _poly_problem(d, n, seed=11):
    f1 = W.Factor("poly", c=(1.0, 0.4, -0.3, 0.2))
    f2 = W.Factor("poly", c=(0.5, -1.0, 0.0, 0.7))
    beta = W.random_unit_vector(d, np.random.default_rng(seed))
    return W.Problem(f"dir d={d} n={n}", d, (n,) * d, beta, 0.1, [W.Term(1.0, (f1,) * d),
                                                                 W.Term(-0.6, (f2,) * d)], tol=1e-12, rmax=20)


def _data(p, op, seed=4):
    """g = u* on the full grid plus a TT that vanishes on the boundary."""
    from paper_2506_04732_gb300 import problem as P
    G = P.full_solution_cores(p, op)
    H = W.random_tt(p.d, p.n[0], [1] + [2] * (p.d - 1) + [1], seed=seed)
    for c in H:
        c[:, 0, :] = 0.0
        c[:, -1, :] = 0.0
    return OT.add(G, H)


CASES = [(1, 9), (2, 8), (3, 7)]


@pytest.mark.parametrize("d,n", CASES)
@pytest.mark.parametrize("cm,co", [(0.0, 1.0), (1.5, 0.4)])
def test_lifted_source_matches_oracle(T, d, n, cm, co):
    from paper_2506_04732_gb300 import problem as P
    p = _poly_problem(d, n)
    op = P.build_operator(p)
    ops = O.build(p)
    G = _data(p, op)
    b = P.source_cores(p, op)
    out = T.TT.empty(list(op.m), 2 * max(OT.ranks(b)) + 4 * max(OT.ranks(G)) + 4)
    T.t2s2_dirichlet_rhs(op, T.TT.from_cores(b), T.TT.from_cores(G), out, 1e-15, 0, cm, co)
    want = DI.lifted_source_tt(ops, O.source_tt(p, ops), G, cm, co)
    assert OT.norm(want) > 1e-2 * OT.norm(b)
    assert OT.diff_norm(out.cores(), want) <= 1e-12 * OT.norm(want)


@pytest.mark.parametrize("d,n", CASES)
def test_solve_matches_dense_full_grid_solve(T, d, n):
    from paper_2506_04732_gb300 import problem as P
    p = _poly_problem(d, n)
    op = P.build_operator(p)
    ops = O.build(p)
    G = _data(p, op)
    b = T.TT.from_cores(P.source_cores(p, op))
    x = T.TT.from_cores([np.ones((1, n - 2, 1))] * d, rcap=40)
    info = T.t2s2_solve_dirichlet(op, b, T.TT.from_cores(G), x, 1e-12, 20, 40)
    assert info.residual <= 1e-12
    ud = DI.dense_solve(ops, O.source_tt(p, ops), G)
    got = OT.full(x.cores())
    assert np.linalg.norm(got - ud) <= 1e-10 * np.linalg.norm(ud)
    # the polynomial u* is the discrete solution
    us = OT.full(O.solution_tt(p, ops))
    assert np.linalg.norm(got - us) <= 1e-10 * np.linalg.norm(us)


def test_zero_data_is_the_plain_solve(T):
    from paper_2506_04732_gb300 import problem as P
    p = W.config0()
    op = P.build_operator(p)
    b = T.TT.from_cores(P.source_cores(p, op))
    m = [v - 2 for v in p.n]
    x1 = T.TT.from_cores([np.ones((1, mm, 1)) for mm in m], rcap=p.rmax + T.RANK_KICK)
    x2 = T.TT.from_cores([np.ones((1, mm, 1)) for mm in m], rcap=p.rmax + T.RANK_KICK)
    i1 = T.t2s2_solve_dirichlet(op, b, None, x1, p.tol, p.rmax, p.max_sweeps)
    i2 = T.t2s2_solve(op, b, x2, p.tol, p.rmax, p.max_sweeps)
    assert i1.residual == i2.residual and x1.r == x2.r
    for c1, c2 in zip(x1.cores(), x2.cores()):
        assert np.array_equal(c1, c2)


def test_bad_data_is_rejected(T):
    from paper_2506_04732_gb300 import problem as P
    p = _poly_problem(2, 8)
    op = P.build_operator(p)
    b = T.TT.from_cores(P.source_cores(p, op))
    interior = T.TT.from_cores(W.random_tt(2, 6, [1, 2, 1], seed=1))   # interior grid, not full
    out = T.TT.empty(list(op.m), 16)
    with pytest.raises(T.T2S2Error) as e:
        T.t2s2_dirichlet_rhs(op, b, interior, out, 1e-12, 0)
    assert e.value.status == 1
    st = T.t2s2_build_spacetime_operator(2, [8, 8], p.beta, p.eps, 5, 1.0)
    gst = T.TT.from_cores(W.random_tt(3, [5, 8, 8], [1, 1, 1, 1], seed=2))
    with pytest.raises(T.T2S2Error):
        T.t2s2_dirichlet_rhs(st, b, gst, out, 1e-12, 0)


def test_full_size_workload_checked_by_oracle(T):
    from paper_2506_04732_gb300 import problem as P
    p = W.config_dirichlet()
    op = P.build_operator(p)
    ops = O.build(p)
    G = _data(p, op, seed=6)
    b = T.TT.from_cores(P.source_cores(p, op))
    x = T.TT.from_cores([np.ones((1, v - 2, 1)) for v in p.n], rcap=p.rmax + T.RANK_KICK + max(OT.ranks(G)))
    info = T.t2s2_solve_dirichlet(op, b, T.TT.from_cores(G), x, p.tol, p.rmax, p.max_sweeps)
    assert info.status == 0 and info.residual <= p.tol
    # the interior equations, recomputed by the oracle: b_g - A (x - g_int)
    bg = DI.lifted_source_tt(ops, O.source_tt(p, ops), G)
    w = OT.add(x.cores(), OT.scale(DI.interior(G), -1.0))
    r = OT.diff_norm(bg, OT.matvec(O.ttm_cores(ops), w)) / OT.norm(bg)
    assert r <= 1.05 * p.tol
    us = O.solution_tt(p, ops)
    assert OT.diff_norm(x.cores(), us) <= 1e-6 * OT.norm(us)
