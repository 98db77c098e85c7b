"""Host logic of the operator build on CPU: the library's per-dimension 1D
collocation matrices (t2s2_dim_matrices, no device involved) against the
oracle's, which are computed by different algorithms (Legendre-Vandermonde
solve and numpy series roots in the oracle; product-form Lagrange
derivatives and bracketed Newton in the library)."""
import numpy as np
import pytest

import paper_2506_04732_gb300 as T
from oracle import collocation as C
from oracle import spacetime as ST


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _close(a, b, rel):
    return np.max(np.abs(a - b)) <= rel * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("n,eps,beta,plain", [
    (5, 0.3, 1.0, False), (16, 1e-2, 0.8, False), (16, 1e-2, -0.8, False),
    (33, 1e-4, 0.57, False), (33, 1e-3, 0.57, True), (12, 0.05, 0.0, False),
    # the extremes of n: one unknown, and the largest operator the library takes
    (3, 0.1, 1.0, False), (3, 1e-6, -1.0, False), (4, 1e-8, 1.0, False),
    (128, 1e-2, 0.7, False), (128, 1e-5, 0.7, False), (128, 1e-3, -0.3, True)])
def test_space_dimension_matches_oracle(n, eps, beta, plain):
    kind = T.DIM_SPACE_PLAIN if plain else T.DIM_SPACE
    got = T.t2s2_dim_matrices(n, eps, beta, kind)
    o = C.op1d(n, eps, beta, plain)
    N = n - 1
    assert _close(got["x"], o.x, 1e-14)
    assert _close(got["eta"], o.eta, 1e-13)
    assert _close(got["Rt"], o.Rt, 1e-12)
    assert _close(got["Lt"], o.Lt, 1e-11)
    cols = [0, N]
    assert _close(got["Rb"], o.R[:, cols], 1e-12)
    assert _close(got["Lb"], beta * o.D[:, cols] - eps * o.D2[:, cols], 1e-11)


@pytest.mark.parametrize("n,T_len", [(3, 1.0), (9, 2.5), (24, 0.4), (128, 0.5)])
def test_time_dimension_matches_oracle(n, T_len):
    got = T.t2s2_dim_matrices(n, 0.0, 2.0 / T_len, T.DIM_TIME)
    o = ST.time_op1d(n, T_len)
    assert _close(got["x"], o.x, 1e-14)
    assert _close(got["eta"], o.g, 1e-14)
    assert _close(got["Rt"], o.Rt, 1e-12)
    assert _close(got["Lt"], o.Lt, 1e-11)
    assert _close(got["Rb"][:, 0], o.r0, 1e-12)
    assert _close(got["Lb"][:, 0], o.l0, 1e-11)


@pytest.mark.parametrize("args", [(2, 0.1, 1.0, 0), (T.MAX_N + 1 if hasattr(T, "MAX_N") else 129, 0.1, 1.0, 0),
                                  (8, 0.1, 1.0, 7), (8, 0.0, 1.0, 0), (8, -1e-3, 1.0, 1),
                                  (8, -1.0, 1.0, 2), (8, float("nan"), 1.0, 0), (8, 0.1, float("inf"), 2)])
def test_invalid_arguments_are_rejected(args):
    with pytest.raises(T.T2S2Error) as e:
        T.t2s2_dim_matrices(*args)
    assert e.value.status == 1
