"""GPU parity of variable coefficients (row N3: beta_k(x_k) and a reaction
rho0 + sum_k rho_k(x_k) + prod_k pi_k(x_k)) against the variable-coefficient
oracle: the rank-2 operator's matrices, solves and CN step; with the product
reaction, the rank-3 apply, the residual, the defect-correction solve against
the dense solve and at full size by the oracle's residual."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import operator as O
from oracle import solve as OS
from oracle import tt as OT
from oracle import varcoef as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2506_04732_gb300 as pkg
    torch.cuda.set_device(0)
    return pkg


def _oracle(vp):
    p = vp.problem
    vc = V.VarCoef(np.asarray(p.beta), [vp.beta_fn(k) for k in range(p.d)], [vp.rho_fn(k) for k in range(p.d)],
                   vp.rho0, [vp.prod_fn(k) for k in range(p.d)] if vp.prod else None)
    return V.build(p, vc)


@pytest.mark.parametrize("d,n", [(1, 9), (3, 9)])
def test_matrices_match_oracle(T, d, n):
    from paper_2506_04732_gb300 import problem as P
    vp = W.config_varcoef(d=d, n=n, ratio=0.02)
    op = P.build_operator_var(vp)
    ops = _oracle(vp)
    for k in range(d):
        _, eta = op.nodes(k)
        assert np.max(np.abs(eta - ops[k].eta)) <= 1e-13
        Rt, Lt = op.matrices(k)
        assert np.max(np.abs(Rt - ops[k].Rt)) <= 1e-11 * np.max(np.abs(ops[k].Rt))
        assert np.max(np.abs(Lt - ops[k].Lt)) <= 1e-11 * np.max(np.abs(ops[k].Lt))


def test_solve_matches_dense(T):
    from paper_2506_04732_gb300 import problem as P
    vp = W.config_varcoef(d=3, n=10, ratio=0.02)
    op = P.build_operator_var(vp)
    ops = _oracle(vp)
    b = T.TT.from_cores(P.varcoef_source_cores(vp, op))
    x = T.TT.from_cores([np.ones((1, 8, 1))] * 3, rcap=40)
    info = T.t2s2_solve(op, b, x, 1e-12, 30, 40)
    assert info.residual <= 1e-12
    xd = OS.dense_solve(ops, V.source_tt(vp.problem, ops))
    assert np.linalg.norm(OT.full(x.cores()) - xd) <= 1e-10 * np.linalg.norm(xd)


def test_cn_step_matches_dense(T):
    from paper_2506_04732_gb300 import problem as P
    vp = W.config_varcoef(d=3, n=10, ratio=0.02)
    op = P.build_operator_var(vp)
    ops = _oracle(vp)
    u0 = O.solution_tt(vp.problem, ops)
    u = T.TT.from_cores(P.solution_cores(vp.problem, op), rcap=24)
    dt = 0.01
    T.t2s2_cn_step(op, u, dt, 1e-12, 16)
    ud = np.linalg.solve(O.dense(ops, 1.0, 0.5 * dt), O.dense(ops, 1.0, -0.5 * dt) @ OT.full(u0).ravel())
    assert np.linalg.norm(OT.full(u.cores()).ravel() - ud) <= 1e-10 * np.linalg.norm(ud)


def test_full_size_workload_checked_by_oracle(T):
    from paper_2506_04732_gb300 import problem as P
    vp = W.config_varcoef()
    p = vp.problem
    op = P.build_operator_var(vp)
    b = T.TT.from_cores(P.varcoef_source_cores(vp, op))
    x = T.TT.from_cores([np.ones((1, v - 2, 1)) for v in p.n], rcap=p.rmax + T.RANK_KICK)
    info = T.t2s2_solve(op, b, x, p.tol, p.rmax, p.max_sweeps)
    assert info.status == 0 and info.residual <= p.tol
    ops = _oracle(vp)
    r = OS.residual(O.ttm_cores(ops), V.source_tt(p, ops), x.cores())
    assert r <= 1.05 * p.tol
    us = O.solution_tt(p, ops)
    assert OT.diff_norm(x.cores(), us) <= 1e-6 * OT.norm(us)


def _prod(d, n, ratio=0.02):
    return W.config_varcoef(d=d, n=n, ratio=ratio, prod=True)


def test_product_reaction_apply_and_residual_match_oracle(T):
    from paper_2506_04732_gb300 import problem as P
    vp = _prod(3, 9)
    op = P.build_operator_var(vp)
    ops = _oracle(vp)
    xc = W.random_tt(3, 7, [1, 3, 4, 1], seed=2)
    x = T.TT.from_cores(xc)
    y = T.TT.empty([7] * 3, 12)
    T.t2s2_apply(op, x, y, 0.4, 1.0)
    assert y.r == [1, 9, 12, 1]
    want = OT.matvec(V.ttm_cores(ops, 0.4, 1.0), xc)
    assert OT.diff_norm(y.cores(), want) <= 1e-12 * OT.norm(want)
    b = V.source_tt(vp.problem, ops)
    res = T.t2s2_residual(op, T.TT.from_cores(b), x)
    want_r = OS.residual(V.ttm_cores(ops), b, xc)
    assert abs(res - want_r) <= 1e-10 * want_r
    # the time steps do not take the product term
    u = T.TT.from_cores(xc, rcap=24)
    with pytest.raises(T.T2S2Error) as e:
        T.t2s2_cn_step(op, u, 1e-2, 1e-10, 16)
    assert e.value.status == 6


def test_product_reaction_solve_matches_dense(T):
    from paper_2506_04732_gb300 import problem as P
    vp = _prod(3, 10)
    op = P.build_operator_var(vp)
    ops = _oracle(vp)
    b = T.TT.from_cores(P.varcoef_source_cores(vp, op))
    x = T.TT.from_cores([np.ones((1, 8, 1))] * 3, rcap=40)
    info = T.t2s2_solve(op, b, x, 1e-11, 30, 60)
    assert info.residual <= 1e-11 and info.refinements >= 1
    bo = V.source_tt(vp.problem, ops)
    xd = np.linalg.solve(V.dense(ops), OT.full(bo).ravel())
    assert np.linalg.norm(OT.full(x.cores()).ravel() - xd) <= 1e-9 * np.linalg.norm(xd)


def test_product_reaction_full_size_checked_by_oracle(T):
    from paper_2506_04732_gb300 import problem as P
    vp = W.config_varcoef(prod=True)
    p = vp.problem
    op = P.build_operator_var(vp)
    b = T.TT.from_cores(P.varcoef_source_cores(vp, op))
    x = T.TT.from_cores([np.ones((1, v - 2, 1)) for v in p.n], rcap=p.rmax + T.RANK_KICK)
    info = T.t2s2_solve(op, b, x, p.tol, p.rmax, p.max_sweeps)
    assert info.status == 0 and info.residual <= p.tol
    print(f"product reaction d=6 n=32: {info.refinements} outer steps, {info.sweeps} sweeps, "
          f"rank {info.max_rank}, residual {info.residual:.2e}")
    ops = _oracle(vp)
    r = OS.residual(V.ttm_cores(ops), V.source_tt(p, ops), x.cores())
    assert r <= 1.05 * p.tol
    us = O.solution_tt(p, ops)
    assert OT.diff_norm(x.cores(), us) <= 1e-6 * OT.norm(us)
