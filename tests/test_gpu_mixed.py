"""GPU parity of the mixed-precision solves (FP64 iterative refinement around
binary32 local solves and BF16 / TF32 tensor-core contractions).

The refinement loop's residual is FP64, so the bar is the FP64 one: the
oracle's residual of the returned solution is <= tol, and on tiny grids the
solution matches the dense LU solve to the accuracy that tol implies.
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


PRECS = ["FP32_REFINE", "TF32_REFINE", "BF16_REFINE"]


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_config0_matches_dense_lu(T, prec):
    p = W.config0()
    op, b, x = _setup(T, p)
    info = T.t2s2_solve(op, b, x, 1e-11, p.rmax, 60, prec=getattr(T, prec))
    assert info.residual <= 1e-11
    assert info.refinements >= 1
    ops = O.build(p)
    ob = O.source_tt(p, ops)
    xd = OS.dense_solve(ops, ob)
    assert OS.residual(O.ttm_cores(ops), ob, x.cores()) <= 1e-11 * 1.01
    assert np.linalg.norm(OT.full(x.cores()) - xd) <= 1e-9 * np.linalg.norm(xd)


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_d5_residual_checked_by_oracle(T, prec):
    p = W.config1(d=5, n=24, ratio=1e-2, rmax=16, tol=1e-8)
    op, b, x = _setup(T, p)
    info = T.t2s2_solve(op, b, x, p.tol, p.rmax, 60, prec=getattr(T, prec))
    ops = O.build(p)
    ob = O.source_tt(p, ops)
    r_or = OS.residual(O.ttm_cores(ops), ob, x.cores())
    assert info.residual <= p.tol
    assert r_or <= p.tol * 1.01
    us = O.solution_tt(p, ops)
    assert OT.diff_norm(x.cores(), us) <= 1e-5 * OT.norm(us)


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_cn_step_matches_dense(T, prec):
    p = W.config2(d=3, n=12, dt=0.01)
    from paper_2506_04732_gb300 import problem as P
    op = P.build_operator(p)
    ops = O.build(p)
    u0 = O.solution_tt(p, ops)
    u = T.TT.from_cores(P.solution_cores(p, op), rcap=16 + T.RANK_KICK)
    info = T.t2s2_cn_step(op, u, p.dt, 1e-11, 16, prec=getattr(T, prec))
    Mp = O.dense(ops, 1.0, 0.5 * p.dt)
    Mm = O.dense(ops, 1.0, -0.5 * p.dt)
    ud = np.linalg.solve(Mp, Mm @ OT.full(u0).ravel())
    assert info.residual <= 1e-11
    assert np.linalg.norm(OT.full(u.cores()).ravel() - ud) <= 1e-9 * np.linalg.norm(ud)


@pytest.mark.parametrize("prec", ["TF32_REFINE", "BF16_REFINE"])
def test_mixed_config1_full_size(T, prec):
    p = W.config1()
    op, b, x = _setup(T, p)
    import time
    torch.cuda.synchronize()
    t = time.time()
    info = T.t2s2_solve(op, b, x, p.tol, p.rmax, p.max_sweeps, prec=getattr(T, prec))
    torch.cuda.synchronize()
    print(f"config1 {prec}: {time.time() - t:.3f}s residual {info.residual:.2e} sweeps {info.sweeps} "
          f"refinements {info.refinements} rank {info.max_rank} local its {info.local_iters}")
    assert info.residual <= p.tol
    ops = O.build(p)
    r_or = OS.residual(O.ttm_cores(ops), O.source_tt(p, ops), x.cores())
    assert r_or <= p.tol * 1.01
    us = O.solution_tt(p, ops)
    assert OT.diff_norm(x.cores(), us) <= 1e-6 * OT.norm(us)
