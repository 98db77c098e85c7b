"""Crank-Nicolson trajectories (eq. ttss-Crank-Nicolson, mass matrix
M = Rt (x) ... (x) Rt) against the oracle, step by step.

* d = 3, n = 16, all 100 steps of dt = 1e-3 against the dense CN recursion
  (the oracle's exact form at that size), in FP64 and with BF16 tensor-core
  contractions under FP64 refinement.
* d = 7, n = 64 (the full Crank-Nicolson workload): the first 10 steps against
  the oracle's own TT trajectory, compared by the accurate difference norm.

Each step rounds its right-hand side at tol and solves to tol, so the error
against an exact trajectory grows by about 2 tol per step; the bounds below
allow ten times that.
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


@pytest.mark.parametrize("prec", ["FP64", "BF16_REFINE"])
def test_100_steps_match_dense_cn_d3(T, prec):
    from paper_2506_04732_gb300 import problem as P
    p = W.config2(d=3, n=16)
    tol = 1e-10
    op = P.build_operator(p)
    ops = O.build(p)
    u = T.TT.from_cores(P.solution_cores(p, op), rcap=p.rmax + T.RANK_KICK)
    Mp = O.dense(ops, 1.0, 0.5 * p.dt)
    Mm = O.dense(ops, 1.0, -0.5 * p.dt)
    step = np.linalg.solve(Mp, Mm)        # the exact CN step as one matrix
    ud = OT.full(O.solution_tt(p, ops)).ravel()
    worst = 0.0
    for k in range(1, p.steps + 1):
        info = T.t2s2_cn_step(op, u, p.dt, tol, p.rmax, prec=getattr(T, prec))
        assert info.residual <= tol
        ud = step @ ud
        err = np.linalg.norm(OT.full(u.cores()).ravel() - ud) / np.linalg.norm(ud)
        worst = max(worst, err)
        assert err <= 20 * k * tol, (k, err)
    print(f"{prec}: worst relative error over 100 steps {worst:.2e}")


def test_first_10_steps_match_oracle_full_size(T):
    from paper_2506_04732_gb300 import problem as P
    p = W.config2()
    op = P.build_operator(p)
    ops = O.build(p)
    u = T.TT.from_cores(P.solution_cores(p, op), rcap=p.rmax + T.RANK_KICK)
    uo = O.solution_tt(p, ops)
    errs = []
    for k in range(1, 11):
        info = T.t2s2_cn_step(op, u, p.dt, p.tol, p.rmax)
        assert info.residual <= p.tol
        uo, res, _ = OS.cn_step(ops, uo, p.dt, p.tol, p.rmax)
        assert res <= p.tol
        errs.append(OT.diff_norm(u.cores(), uo) / OT.norm(uo))
        assert errs[-1] <= 20 * k * p.tol, (k, errs)
    print("per-step relative difference to the oracle:", " ".join(f"{e:.1e}" for e in errs))
