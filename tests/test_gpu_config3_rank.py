"""The instances of the 256-instance d = 5 workload (seeds 1000 + i) whose
best rank-16 approximation does not reach 1e-8.  Twelve of them stop above
1e-8 under the solver's rank cap of 16; four (21, 116, 145, 210) reach it
because the sweep's iterates carry up to rmax + kick = 24 ranks.

All of them have n = 16 (14 unknowns per dimension) and diffusion ratios
eps/|beta L| between 1.2e-4 and 6e-3: thin layers that 16 nodes resolve only
roughly, with discrete solutions of high TT rank.  For each seed the test
shows, with the oracle's residual of the original collocation system, that

* a tight GPU solve at a generous rank cap is close to the discrete
  solution (oracle residual <= 5e-9);
* its best rank-16 approximation in the SVD sense (the oracle's rounding
  with cap 16) leaves a residual above 1e-8 and above ten times the tight
  solve's: rank 16 alone cannot reach the tolerance, the solver is not what
  falls short;
* the GPU solver reaches 1e-8 once its cap is raised to 40.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import operator as O
from oracle import solve as OS
from oracle import tt as OT

pytestmark = pytest.mark.gpu

# seeds i of W.config3(i) whose rank-16 solutions stay above 1e-8 (145 hovers
# at 1.1e-8 - 1.5e-8 under the cap and crosses 1e-8 after nine sweeps in some
# summation orders, not in others)
RANK_CAPPED = [13, 21, 47, 51, 60, 88, 101, 116, 142, 145, 148, 154, 187, 205, 210, 213]


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2506_04732_gb300 as pkg
    torch.cuda.set_device(0)
    return pkg


def _solve(T, op, b, p, tol, rmax, sweeps):
    x = T.TT.from_cores([np.ones((1, n - 2, 1)) for n in p.n], rcap=rmax + T.RANK_KICK)
    info = T.t2s2_solve(op, b, x, tol, rmax, sweeps, allow_noconv=True)
    return x, info


@pytest.mark.parametrize("i", RANK_CAPPED)
def test_rank_cap_16_is_what_stops_the_instance(T, i):
    from paper_2506_04732_gb300 import problem as P
    p = W.config3(i)
    assert p.n[0] == 16 and p.ratio < 1e-2
    op = P.build_operator(p)
    b = T.TT.from_cores(P.source_cores(p, op))
    ops = O.build(p)
    A, ob = O.ttm_cores(ops), O.source_tt(p, ops)
    # the discrete solution, to a tight tolerance at a generous cap
    xt, _ = _solve(T, op, b, p, 1e-10, 48, 60)
    xt = xt.cores()
    r_t = OS.residual(A, ob, xt)
    assert r_t <= 5e-9
    # no rank-16 truncation of it reaches the tolerance, and what it misses
    # comes from the truncation (ten times the tight solve's own residual)
    x16 = OT.round_tt(xt, 0.0, 16)
    assert max(OT.ranks(x16)) <= 16
    r16 = OS.residual(A, ob, x16)
    assert r16 > 1e-8 and r16 > 10 * r_t
    # with a cap of 40 the solver reaches it (checked by the oracle)
    x40, info = _solve(T, op, b, p, 1e-8, 40, 50)
    assert info.status == 0
    assert OS.residual(A, ob, x40.cores()) <= 1.01e-8


def test_solve_stops_early_at_the_rank_cap(T):
    """Under the cap of 16 a rank-capped instance stops once its ranks sit at
    rmax + kick and its residual has not halved in 8 sweeps: T2S2_ENOCONV well
    before the 50-sweep cap, with the last iterate and its residual."""
    from paper_2506_04732_gb300 import problem as P
    p = W.config3(13)
    op = P.build_operator(p)
    b = T.TT.from_cores(P.source_cores(p, op))
    x, info = _solve(T, op, b, p, 1e-8, 16, 50)
    assert info.status == 4 and info.residual > 1e-8
    assert info.sweeps < 20 and info.max_rank == 16 + T.RANK_KICK
    ops = O.build(p)
    r = OS.residual(O.ttm_cores(ops), O.source_tt(p, ops), x.cores())
    assert abs(r - info.residual) <= 1e-3 * info.residual
