"""Direct pins of oracle helpers that the other pins reach only through their
callers: the truncation rank of TT-SVD (Methods, rounding with a per-unfolding
threshold), the Legendre table behind the GLL and superconsistent points
(Overview (i)-(ii)), the exact TT of separable data (Methods), and the
Crank-Nicolson right-hand side (eq. ttss-Crank-Nicolson)."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import workloads as W
from oracle import gll as G
from oracle import operator as O
from oracle import solve as S
from oracle import tt as T


def _brute_trunc_rank(s, delta, rmax=None):
    # smallest r >= 1 whose discarded tail s[r:] has 2-norm <= delta
    for r in range(1, len(s) + 1):
        if np.sqrt(np.sum(s[r:] ** 2)) <= delta:
            break
    if rmax is not None:
        r = min(r, rmax)
    return max(r, 1)


@pytest.mark.parametrize("seed", range(20))
def test_trunc_rank_is_the_smallest_rank_meeting_the_tail_bound(seed):
    rng = np.random.default_rng(seed)
    s = np.sort(rng.random(12) ** 3)[::-1]
    delta = rng.uniform(0.0, np.linalg.norm(s))
    assert T.trunc_rank(s, delta) == _brute_trunc_rank(s, delta)
    assert T.trunc_rank(s, delta, rmax=3) == _brute_trunc_rank(s, delta, rmax=3)


def test_trunc_rank_limits():
    s = np.array([3.0, 2.0, 1.0, 0.5])
    assert T.trunc_rank(s, 0.0) == 4                 # nothing may be dropped
    assert T.trunc_rank(s, np.linalg.norm(s)) == 1   # never below rank 1
    assert T.trunc_rank(s, 0.6) == 3                 # the tail [0.5] is within 0.6
    assert T.trunc_rank(s, 1.2) == 2                 # |[1, 0.5]| = 1.118 <= 1.2
    # a tail equal to delta is a tie, and a tie keeps the larger rank
    assert T.trunc_rank(s, 0.5) == 4


@pytest.mark.parametrize("N", [1, 2, 7, 12])
def test_legendre_table_matches_numpy_legendre_series(N):
    rng = np.random.default_rng(N)
    x = np.concatenate([[-1.0, 1.0, 0.0], rng.uniform(-1, 1, 9)])
    P, D, S2 = G.legendre_table(N, x)
    for k in range(N + 1):
        e = np.zeros(k + 1)
        e[k] = 1.0
        scale = max(1.0, k ** 4)
        assert np.allclose(P[:, k], npleg.legval(x, e), rtol=0, atol=1e-13)
        assert np.allclose(D[:, k], npleg.legval(x, npleg.legder(e)), rtol=0, atol=1e-13 * scale)
        assert np.allclose(S2[:, k], npleg.legval(x, npleg.legder(e, 2)), rtol=0, atol=1e-13 * scale)


@pytest.mark.parametrize("d", [1, 2, 4])
def test_separable_tt_is_the_sum_of_outer_products(d):
    rng = np.random.default_rng(10 + d)
    n = [3, 4, 2, 5][:d]
    terms = 3
    vecs = [[rng.standard_normal(n[k]) for k in range(d)] for _ in range(terms)]
    coefs = rng.standard_normal(terms)
    want = 0.0
    for t in range(terms):
        out = vecs[t][0]
        for k in range(1, d):
            out = np.multiply.outer(out, vecs[t][k])
        want = want + coefs[t] * out
    cores = O.separable_tt(vecs, coefs)
    assert np.allclose(T.full(cores), want, rtol=0, atol=1e-13)
    if d > 1:
        assert T.ranks(cores)[1:-1] == [terms] * (d - 1)


def test_cn_rhs_is_mass_minus_half_step_operator():
    p = W.config2(d=3, n=7, dt=0.01)
    ops = O.build(p)
    m = [n - 2 for n in p.n]
    u = W.random_tt(p.d, m, [1, 2, 3, 1], seed=3)
    dt = 0.01
    got = T.full(S.cn_rhs(ops, u, dt, 1e-15, 50)).ravel()
    uf = T.full(u).ravel()
    want = O.dense(ops, 1.0, 0.0) @ uf - 0.5 * dt * (O.dense(ops, 0.0, 1.0) @ uf)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
