"""GPU parity of the unified space-time form (time as the first collocated
dimension, the initial condition lifted into the right-hand side; Methods
overview, Results "Global Accuracy and Computational Cost") against the
space-time oracle.

* the time dimension's nodes and matrices, and the spatial ones behind it;
* the lifted right-hand side b - L0 (x) M_x u0 - R0 (x) A_x u0 against the
  oracle's lifted source, including the one-spatial-dimension case (the
  single-core apply);
* the solve against the oracle's dense solve to 1e-10 relative (FP64);
* at the full size of the space-time workload (d = 5 plus time, n = 32,
  n_t = 24): the oracle recomputes the residual of the GPU solution, and the
  solution lies within 1e-6 of the manufactured u*.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import solve as OS
from oracle import spacetime as ST
from oracle import tt as OT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2506_04732_gb300 as pkg
    torch.cuda.set_device(0)
    return pkg


def _st(d, n, n_t, T_len, ratio=0.02, seed=3):
    beta = W.random_unit_vector(d, np.random.default_rng(seed))
    terms = [W.Term(1.0, (W.Factor("sine", m=1),) * d), W.Term(-0.4, (W.Factor("wsine", m=2),) * d)]
    sp = W.Problem(f"st d={d}", d, (n,) * d, beta, ratio * W.EDGE_LENGTH, terms, tol=1e-12, rmax=30)
    return ST.SpaceTimeProblem(sp, (W.Factor("exp", m=0.8), W.Factor("poly", c=(1.0, 0.5, -0.2))), n_t, T_len)


def _op(T, st):
    sp = st.space
    return T.t2s2_build_spacetime_operator(sp.d, sp.n, sp.beta, sp.eps, st.n_t, st.T, sp.plain_sc)


def _rhs(T, st, op, tol=1e-14, rmax=0):
    from paper_2506_04732_gb300 import problem as P
    dims = P.spacetime_dims(st)
    b = T.TT.from_cores(P.spacetime_source_cores(st, dims))
    u0 = T.TT.from_cores(P.spacetime_initial_cores(st, dims))
    cap = 2 * max(b.r) + 4 * max(u0.r) + 8
    rhs = T.TT.empty(list(op.m), cap)
    T.t2s2_spacetime_rhs(op, b, u0, rhs, tol, rmax)
    return rhs


CASES = [(1, 9, 5, 1.0), (2, 8, 6, 2.5), (3, 7, 4, 0.3)]


@pytest.mark.parametrize("d,n,n_t,T_len", CASES)
def test_nodes_and_matrices_match_oracle(T, d, n, n_t, T_len):
    st = _st(d, n, n_t, T_len)
    op = _op(T, st)
    top, ops = ST.build(st)
    assert op.d == d + 1 and op.m[0] == n_t - 1
    x, g = op.nodes(0)
    assert np.max(np.abs(x - top.x)) <= 1e-14 and np.max(np.abs(g - top.g)) <= 1e-14
    Rt, Lt = op.matrices(0)
    assert np.max(np.abs(Rt - top.Rt)) <= 1e-12 * np.max(np.abs(top.Rt))
    assert np.max(np.abs(Lt - top.Lt)) <= 1e-12 * np.max(np.abs(top.Lt))
    for k in range(d):
        xk, ek = op.nodes(k + 1)
        assert np.max(np.abs(xk - ops[k].x)) <= 1e-14 and np.max(np.abs(ek - ops[k].eta)) <= 1e-13
        Rk, Lk = op.matrices(k + 1)
        assert np.max(np.abs(Rk - ops[k].Rt)) <= 1e-11 * np.max(np.abs(ops[k].Rt))
        assert np.max(np.abs(Lk - ops[k].Lt)) <= 1e-11 * np.max(np.abs(ops[k].Lt))


@pytest.mark.parametrize("d,n,n_t,T_len", CASES)
def test_lifted_rhs_matches_oracle(T, d, n, n_t, T_len):
    st = _st(d, n, n_t, T_len)
    op = _op(T, st)
    top, ops = ST.build(st)
    rhs = _rhs(T, st, op)
    want = ST.lifted_source_tt(st, top, ops)
    assert OT.diff_norm(rhs.cores(), want) <= 1e-12 * OT.norm(want)
    # the lifting is not a no-op: the initial condition changes the source
    assert OT.diff_norm(ST.source_tt(st, top, ops), want) > 1e-3 * OT.norm(want)


@pytest.mark.parametrize("d,n,n_t,T_len", CASES)
def test_solve_matches_dense_solve(T, d, n, n_t, T_len):
    st = _st(d, n, n_t, T_len)
    op = _op(T, st)
    top, ops = ST.build(st)
    rhs = _rhs(T, st, op)
    x = T.TT.from_cores([np.ones((1, m, 1)) for m in op.m], rcap=30 + T.RANK_KICK)
    info = T.t2s2_solve(op, rhs, x, 1e-12, 30, 40)
    assert info.residual <= 1e-12
    ud = ST.dense_solve(st, top, ops)
    assert np.linalg.norm(OT.full(x.cores()) - ud) <= 1e-10 * np.linalg.norm(ud)


def test_rhs_rejects_a_bad_output(T):
    st = _st(2, 8, 6, 1.0)
    op = _op(T, st)
    from paper_2506_04732_gb300 import problem as P
    dims = P.spacetime_dims(st)
    b = T.TT.from_cores(P.spacetime_source_cores(st, dims))
    u0 = T.TT.from_cores(P.spacetime_initial_cores(st, dims))
    bad_loc = T.TT.empty(list(op.m), 16)
    bad_loc.loc = 5
    with pytest.raises(T.T2S2Error) as e:
        T.t2s2_spacetime_rhs(op, b, u0, bad_loc, 1e-12, 16)
    assert e.value.status == 1
    m = list(op.m)
    m[1] += 1
    with pytest.raises(T.T2S2Error) as e:
        T.t2s2_spacetime_rhs(op, b, u0, T.TT.empty(m, 16), 1e-12, 16)
    assert e.value.status == 1
    # a spatial operator is not a space-time one
    sop = T.t2s2_build_operator(2, [8, 8], st.space.beta, st.space.eps)
    with pytest.raises(T.T2S2Error):
        T.t2s2_spacetime_rhs(sop, b, u0, T.TT.empty(list(op.m), 16), 1e-12, 16)


def test_full_size_workload_residual_checked_by_oracle(T):
    st = W.config_spacetime()
    sp = st.space
    op = _op(T, st)
    rhs = _rhs(T, st, op, tol=1e-2 * sp.tol, rmax=0)
    x = T.TT.from_cores([np.ones((1, m, 1)) for m in op.m], rcap=sp.rmax + T.RANK_KICK)
    info = T.t2s2_solve(op, rhs, x, sp.tol, sp.rmax, sp.max_sweeps)
    assert info.status == 0 and info.residual <= sp.tol
    top, ops = ST.build(st)
    b_or = ST.lifted_source_tt(st, top, ops)
    r_or = OS.residual(ST.ttm_cores(top, ops), b_or, x.cores())
    assert r_or <= 1.05 * sp.tol
    us = ST.solution_tt(st, top, ops)
    assert OT.diff_norm(x.cores(), us) <= 1e-6 * OT.norm(us)
