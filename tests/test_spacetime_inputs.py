"""Host-side inputs of the space-time form (row N1) on CPU: the source and the
initial condition sampled at the nodes the library reports
(t2s2_dim_matrices) against the space-time oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import spacetime as ST
from oracle import tt as OT


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _st(d, n, n_t, T_len):
    beta = W.random_unit_vector(d, np.random.default_rng(3))
    terms = [W.Term(1.0, (W.Factor("sine", m=1),) * d), W.Term(-0.4, (W.Factor("wsine", m=2),) * d)]
    sp = W.Problem(f"st d={d}", d, (n,) * d, beta, 2e-2, terms, tol=1e-10, rmax=20)
    return ST.SpaceTimeProblem(sp, (W.Factor("exp", m=0.8), W.Factor("poly", c=(1.0, 0.5, -0.2))), n_t, T_len)


@pytest.mark.parametrize("d,n,n_t,T_len", [(1, 9, 5, 1.0), (2, 8, 6, 2.5), (3, 7, 4, 0.3)])
def test_spacetime_inputs_match_oracle(d, n, n_t, T_len):
    from paper_2506_04732_gb300 import problem as P
    st = _st(d, n, n_t, T_len)
    dims = P.spacetime_dims(st)
    top, ops = ST.build(st)
    b = OT.full(P.spacetime_source_cores(st, dims))
    want = OT.full(ST.source_tt(st, top, ops))
    assert np.max(np.abs(b - want)) <= 1e-12 * np.max(np.abs(want))
    u0 = OT.full(P.spacetime_initial_cores(st, dims))
    assert np.max(np.abs(u0 - OT.full(ST.initial_tt(st, ops)))) <= 1e-14 * np.max(np.abs(u0))
