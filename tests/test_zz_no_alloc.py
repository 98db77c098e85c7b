"""t2s2_norm_noalloc: the TT norm for callers that cannot allocate device memory.

Such callers (real-time loops whose memory is fixed at start-up, hosts whose
framework allocator owns the device) get the same accurate norm as t2s2_norm,
with all temporaries in the library's static device array.  Checked against
the FP64 oracle's orthogonalised norm and against t2s2_norm, on two calls in a
row, with the device's free memory unchanged across the calls.  This file is
collected last so that a failure here does not hide any other test.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import tt as OT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2506_04732_gb300 as pkg
    torch.cuda.set_device(0)
    return pkg


def test_noalloc_norm_matches_oracle_and_norm_on_two_calls_in_a_row(T):
    from paper_2506_04732_gb300 import problem as P
    p = W.config1(d=6, n=32)
    op = P.build_operator(p)
    trains = [W.random_tt(6, 30, [1, 7, 12, 20, 9, 4, 1], seed=s) for s in (1, 2)]
    xs = [T.TT.from_cores(c) for c in trains]
    T.t2s2_norm_noalloc(xs[0])          # first call on the device: address look-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got = [T.t2s2_norm_noalloc(x) for x in xs]   # two calls in a row share the array
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0  # nothing was allocated
    for c, x, g in zip(trains, xs, got):
        want = OT.norm(c)
        assert abs(g - want) <= 1e-13 * want
        assert abs(g - T.t2s2_norm(op, x)) <= 1e-13 * want
    # an exactly rank-deficient train (x - x) too
    c = W.random_tt(4, 16, [1, 3, 5, 2, 1], seed=3)
    z = T.TT.from_cores(OT.add(c, OT.scale(c, -1.0)))
    assert T.t2s2_norm_noalloc(z) <= 1e-13 * OT.norm(c)


def test_noalloc_uneven_ranks_near_the_limit(T):
    # interior cores of the train's copy are padded to the largest rank on
    # both sides: either the size check rejects the train up front, or the
    # norm is right
    c = W.random_tt(4, 126, [1, 2, 96, 2, 1], seed=5)
    x = T.TT.from_cores(c)
    try:
        got = T.t2s2_norm_noalloc(x)
    except T.T2S2Error as e:
        assert e.status == 2
        return
    want = OT.norm(c)
    assert abs(got - want) <= 1e-13 * want
    # the next call still works on the shared array
    small = W.random_tt(3, 8, [1, 2, 2, 1], seed=6)
    assert abs(T.t2s2_norm_noalloc(T.TT.from_cores(small)) - OT.norm(small)) <= 1e-13 * OT.norm(small)


def test_noalloc_rejects_trains_beyond_the_static_array(T):
    big = T.TT.empty([126] * 3, 96, ranks=[1, 96, 96, 1])
    with pytest.raises(T.T2S2Error) as e:
        T.t2s2_norm_noalloc(big)
    assert e.value.status == 2
    host = T.TT.from_cores(W.random_tt(3, 8, [1, 2, 2, 1], seed=4), device="cpu")
    with pytest.raises(T.T2S2Error) as e:
        T.t2s2_norm_noalloc(host)
    assert e.value.status == 1
