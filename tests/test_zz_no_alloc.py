"""t2s2_norm_noalloc: the TT norm for callers that cannot allocate device memory.

Such callers (graph capture, fixed-memory real-time loops, hosts whose
allocator owns the device) get the same accurate norm as t2s2_norm, with all
temporaries in the library's static device array.  This file is collected last
so that a failure here does not hide any other test.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2506_04732_gb300 as pkg
    torch.cuda.set_device(0)
    return pkg


def test_noalloc_norm_matches_norm_on_two_calls_in_a_row(T):
    from paper_2506_04732_gb300 import problem as P
    p = W.config1(d=6, n=32)
    op = P.build_operator(p)
    for seed in (1, 2):   # two calls in a row share (and reuse) the static array
        x = T.TT.from_cores(W.random_tt(6, 30, [1, 7, 12, 20, 9, 4, 1], seed=seed))
        ref = T.t2s2_norm(op, x)
        got = T.t2s2_norm_noalloc(x)
        assert abs(got - ref) <= 1e-13 * ref
    # an exactly rank-deficient train (x - x) too
    c = W.random_tt(4, 16, [1, 3, 5, 2, 1], seed=3)
    from oracle import tt as OT
    z = T.TT.from_cores(OT.add(c, OT.scale(c, -1.0)))
    assert T.t2s2_norm_noalloc(z) <= 1e-13 * OT.norm(c)


def test_noalloc_rejects_trains_beyond_the_static_array(T):
    big = T.TT.empty([126] * 3, 96, ranks=[1, 96, 96, 1])
    with pytest.raises(T.T2S2Error) as e:
        T.t2s2_norm_noalloc(big)
    assert e.value.status == 2
    host = T.TT.from_cores(W.random_tt(3, 8, [1, 2, 2, 1], seed=4), device="cpu")
    with pytest.raises(T.T2S2Error) as e:
        T.t2s2_norm_noalloc(host)
    assert e.value.status == 1
