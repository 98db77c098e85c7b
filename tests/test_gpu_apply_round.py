"""GPU parity: 1D matrices, TT apply, rounding, norms and residuals against the oracle.

Tolerances: FP64 everywhere; apply and norms match to 1e-12 relative (a few
ulps times the contraction length), rounding is compared through the full
tensors (gauges differ) against its own error bound.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import operator as O
from oracle import tt as OT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2506_04732_gb300 as pkg
    torch.cuda.set_device(0)
    return pkg


def _op(T, p):
    from paper_2506_04732_gb300 import problem as P
    return P.build_operator(p), O.build(p)


CASES = [W.config0(), W.config1(d=3, n=10), W.config1(d=4, n=33), W.config3(0), W.config3(5),
         W.config2(d=3, n=64)]


@pytest.mark.parametrize("p", CASES, ids=lambda p: p.name)
def test_nodes_and_matrices_match_oracle(T, p):
    op, ops = _op(T, p)
    for k in range(p.d):
        x, eta = op.nodes(k)
        assert np.max(np.abs(x - ops[k].x)) < 1e-14
        assert np.max(np.abs(eta - ops[k].eta)) < 1e-13
        Rt, Lt = op.matrices(k)
        assert np.max(np.abs(Rt - ops[k].Rt)) < 1e-11 * max(1, np.abs(ops[k].Rt).max())
        assert np.max(np.abs(Lt - ops[k].Lt)) < 1e-11 * np.abs(ops[k].Lt).max()


def test_plain_switch(T):
    p = W.config0()
    p.plain_sc = True
    op, ops = _op(T, p)
    x, eta = op.nodes(1)
    assert np.allclose(eta, x[1:-1], atol=0, rtol=0)


APPLY = [
    (3, 14, [1, 3, 4, 1]),
    (6, 30, [1, 5, 7, 20, 9, 3, 1]),      # ragged ranks, 2m = 60 < 64 rows
    (4, 31, [1, 33, 70, 65, 1]),          # ranks beyond one 64-wide tile
    (5, 46, [1, 16, 16, 16, 16, 1]),      # 2m = 92: two row tiles
    (2, 62, [1, 40, 1]),
    (1, 20, [1, 1]),
]


@pytest.mark.parametrize("d,m,r", APPLY)
@pytest.mark.parametrize("cm,co", [(0.0, 1.0), (1.0, -0.05), (1.0, 0.5)])
def test_apply_matches_oracle(T, d, m, r, cm, co):
    p = W.config1(d=d, n=m + 2, ratio=3e-3)
    op, ops = _op(T, p)
    x = W.random_tt(d, m, r, seed=d * 100 + m)
    tx = T.TT.from_cores(x)
    ty = T.TT.empty(tx.m, 2 * max(r))
    T.t2s2_apply(op, tx, ty, c_mass=cm, c_op=co)
    assert ty.r == [1] + [2 * v for v in r[1:-1]] + [1]
    ref = OT.matvec(O.ttm_cores(ops, cm, co), x)
    # cores are built exactly, so compare core by core
    for a, b in zip(ty.cores(), ref):
        assert a.shape == b.shape
        assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.abs(b).max())


def test_apply_host_buffers(T):
    p = W.config1(d=4, n=20)
    op, ops = _op(T, p)
    x = W.random_tt(4, 18, [1, 3, 5, 2, 1], seed=3)
    tx = T.TT.from_cores(x, device="cpu")
    ty = T.TT.empty(tx.m, 10, device="cpu")
    T.t2s2_apply(op, tx, ty)
    ref = OT.matvec(O.ttm_cores(ops), x)
    assert OT.diff_norm(ty.cores(), ref) <= 1e-13 * OT.norm(ref)


@pytest.mark.parametrize("d,m,r,tol", [(3, 14, [1, 6, 9, 1], 1e-10), (5, 30, [1, 12, 20, 17, 8, 1], 1e-6),
                                       (4, 62, [1, 40, 80, 40, 1], 1e-8), (6, 8, [1, 8, 30, 40, 30, 8, 1], 1e-4),
                                       (2, 5, [1, 3, 1], 1e-12)])
def test_round_error_bound_and_ranks(T, d, m, r, tol):
    p = W.config1(d=d, n=m + 2)
    op, _ = _op(T, p)
    # a TT with redundant rank: sum of a low-rank TT and a small perturbation
    base = W.random_tt(d, m, [1] + [min(v, 4) for v in r[1:-1]] + [1], seed=7)
    noise = W.random_tt(d, m, r, seed=8)
    x = OT.add(base, OT.scale(noise, 1e-3))
    tx = T.TT.from_cores(x)
    T.t2s2_round(op, tx, tol)
    y = tx.cores()
    err = OT.diff_norm(y, x) / OT.norm(x)
    assert err <= tol * (1 + 1e-8)
    # ranks agree with the oracle's rounding except at singular-value ties
    ref = OT.round_tt(x, tol)
    for a, b in zip(OT.ranks(y), OT.ranks(ref)):
        assert abs(a - b) <= 1
    assert OT.diff_norm(y, ref) <= 2 * tol * OT.norm(x)


def test_round_with_cap(T):
    p = W.config1(d=4, n=22)
    op, _ = _op(T, p)
    x = W.random_tt(4, 20, [1, 12, 15, 10, 1], seed=9)
    tx = T.TT.from_cores(x)
    T.t2s2_round(op, tx, 1e-14, rmax=5)
    assert max(tx.r) <= 5
    ref = OT.round_tt(x, 1e-14, 5)
    assert OT.diff_norm(tx.cores(), ref) <= 1e-8 * OT.norm(x)


def test_round_exact_low_rank(T):
    # duplicated rank-1 cores (rank 2 by construction) round back to rank 1
    p = W.config1(d=5, n=12)
    op, _ = _op(T, p)
    rng = np.random.default_rng(1)
    x = [rng.standard_normal((1, 10, 1)) for _ in range(5)]
    xx = OT.add(x, OT.scale(x, 0.5))
    tx = T.TT.from_cores(xx)
    T.t2s2_round(op, tx, 1e-12)
    assert tx.r == [1] * 6
    assert OT.diff_norm(tx.cores(), OT.scale(x, 1.5)) <= 1e-13 * OT.norm(x)


def _cancelling_train(d, m, r, seed, scale=1e3):
    """t1 - t1 + 1e-12 t2 + t3 as one train of rank 4r (an exactly cancelling
    pair and a part at 1e-12 ahead of the dominant part, the structure of
    b - A x near convergence), with the norm moved from the first core to the
    last."""
    t1 = W.random_tt(d, m, [1] + [r] * (d - 1) + [1], seed=seed)
    t2 = W.random_tt(d, m, [1] + [r] * (d - 1) + [1], seed=seed + 1)
    t3 = W.random_tt(d, m, [1] + [r] * (d - 1) + [1], seed=seed + 2)
    x = OT.add(OT.add(OT.add(t1, OT.scale(t1, -1.0)), OT.scale(t2, 1e-12)), t3)
    x[0] = x[0] / scale
    x[-1] = x[-1] * scale
    return x, t3


@pytest.mark.parametrize("seed", [11, 12])
def test_round_keeps_a_train_with_a_cancelling_pair(T, seed):
    # Methods, TT rounding: the orthogonalisation must represent the train to
    # working precision however rank-deficient its unfoldings are; a plain
    # second CholeskyQR pass that zeroed small pivots in column order lost
    # ~1e-12 of such a train (up to 1e-6 on solver right-hand sides)
    p = W.config1(d=6, n=32)
    op, _ = _op(T, p)
    x, t3 = _cancelling_train(6, 30, 8, seed)
    tx = T.TT.from_cores(x)
    T.t2s2_round(op, tx, 0.0)
    assert OT.diff_norm(tx.cores(), x) <= 1e-13 * OT.norm(x)
    tx = T.TT.from_cores(x)
    T.t2s2_round(op, tx, 1e-10)
    assert max(tx.r) <= 8
    assert OT.diff_norm(tx.cores(), t3) <= 1e-10 * OT.norm(t3)


def test_norm_and_residual(T):
    p = W.config1(d=4, n=18)
    op, ops = _op(T, p)
    x = W.random_tt(4, 16, [1, 4, 6, 3, 1], seed=11)
    b = W.random_tt(4, 16, [1, 2, 2, 2, 1], seed=12)
    tx, tb = T.TT.from_cores(x), T.TT.from_cores(b)
    assert abs(T.t2s2_norm(op, tx) - OT.norm(x)) <= 1e-13 * OT.norm(x)
    res = T.t2s2_residual(op, tb, tx)
    ref = OT.diff_norm(b, OT.matvec(O.ttm_cores(ops), x)) / OT.norm(b)
    assert abs(res - ref) <= 1e-12 * ref
    res2 = T.t2s2_residual(op, tb, tx, c_mass=1.0, c_op=0.01)
    ref2 = OT.diff_norm(b, OT.matvec(O.ttm_cores(ops, 1.0, 0.01), x)) / OT.norm(b)
    assert abs(res2 - ref2) <= 1e-12 * ref2


def test_errors_are_status_codes(T):
    with pytest.raises(T.T2S2Error) as e:
        T.t2s2_build_operator(3, [2, 5, 5], [1, 1, 1], 0.1)
    assert e.value.status == 1
    with pytest.raises(T.T2S2Error):
        T.t2s2_build_operator(3, [5, 5, 5], [1, 1, 1], -0.1)
    p = W.config1(d=3, n=10)
    op, _ = _op(T, p)
    x = T.TT.from_cores(W.random_tt(3, 8, [1, 4, 4, 1], seed=1))
    small = T.TT.empty(x.m, 2)           # too small for rank 8 output
    with pytest.raises(T.T2S2Error) as e:
        T.t2s2_apply(op, x, small)
    assert e.value.status == 2


def test_rank_deficient_orthogonalisation_is_finite(T):
    # TT sums whose stored ranks exceed their true ranks (x - x, 2x = x + x,
    # b - A x with b = A x) must orthogonalise without NaN / Inf.
    p = W.config1(d=4, n=14)
    op, ops = _op(T, p)
    x = W.random_tt(4, 12, [1, 3, 5, 2, 1], seed=21)
    zero = OT.add(x, OT.scale(x, -1.0))
    assert T.t2s2_norm(op, T.TT.from_cores(zero)) <= 1e-13 * OT.norm(x)
    two = T.TT.from_cores(OT.add(x, x))
    assert abs(T.t2s2_norm(op, two) - 2 * OT.norm(x)) <= 1e-13 * OT.norm(x)
    T.t2s2_round(op, two, 1e-12)
    assert OT.ranks(two.cores()) == OT.ranks(OT.round_tt(x, 1e-12))
    assert OT.diff_norm(two.cores(), OT.scale(x, 2.0)) <= 1e-12 * OT.norm(x)
    b = OT.matvec(O.ttm_cores(ops, 1.0, 0.3), x)
    r = T.t2s2_residual(op, T.TT.from_cores(b), T.TT.from_cores(x), c_mass=1.0, c_op=0.3)
    assert np.isfinite(r) and r <= 1e-13


def test_diff_norm_resolves_tiny_differences(T):
    # x and y agree to ~1e-10 relative: the TT difference still gives the
    # distance to a few digits (the dot-product formula would return noise)
    from paper_2506_04732_gb300 import problem as P
    p = W.config1(d=4, n=12)
    op = P.build_operator(p)
    x = W.random_tt(4, 10, [1, 3, 4, 2, 1], seed=11)
    y = [c.copy() for c in x]
    y[2] = y[2] + 1e-10 * np.random.default_rng(3).standard_normal(y[2].shape)
    d_gpu = T.t2s2_diff_norm(op, T.TT.from_cores(x), T.TT.from_cores(y))
    d_or = OT.diff_norm(x, y)
    assert d_or > 0
    assert abs(d_gpu - d_or) <= 1e-5 * d_or
    assert T.t2s2_diff_norm(op, T.TT.from_cores(x), T.TT.from_cores(x)) <= 1e-14 * OT.norm(x)


@pytest.mark.parametrize("scale", [1e-3, 1e-7, 1e-9])
def test_residual_resolves_small_residuals(T, scale):
    # b = A x + scale * e: the residual is ~scale, many orders below |b|; the
    # library's double-double <z, z> must still give it to five digits (FP64
    # dot products would return noise below ~1e-8)
    p = W.config1(d=4, n=14)
    op, ops = _op(T, p)
    x = W.random_tt(4, 12, [1, 3, 5, 2, 1], seed=31)
    e = W.random_tt(4, 12, [1, 2, 2, 2, 1], seed=32)
    A = O.ttm_cores(ops, 1.0, 0.3)
    ax = OT.matvec(A, x)
    b = OT.add(ax, OT.scale(e, scale * OT.norm(ax) / OT.norm(e)))
    got = T.t2s2_residual(op, T.TT.from_cores(b), T.TT.from_cores(x), c_mass=1.0, c_op=0.3)
    ref = np.linalg.norm(OT.full(b) - OT.full(ax)) / np.linalg.norm(OT.full(b))
    assert abs(got - ref) <= 1e-5 * ref


def test_residual_near_the_rounding_floor(T):
    # a residual of ~1e-12 |b|: the double-double norm must still resolve it
    # (the binary64 evaluation of A x itself is good to ~4e-15 here)
    p = W.config1(d=4, n=14)
    op, ops = _op(T, p)
    x = W.random_tt(4, 12, [1, 3, 5, 2, 1], seed=41)
    e = W.random_tt(4, 12, [1, 2, 2, 2, 1], seed=42)
    A = O.ttm_cores(ops, 1.0, 0.3)
    ax = OT.matvec(A, x)
    b = OT.add(ax, OT.scale(e, 1e-12 * OT.norm(ax) / OT.norm(e)))
    got = T.t2s2_residual(op, T.TT.from_cores(b), T.TT.from_cores(x), c_mass=1.0, c_op=0.3)
    ref = np.linalg.norm(OT.full(b) - OT.full(ax)) / np.linalg.norm(OT.full(b))
    assert abs(got - ref) <= 1e-2 * ref
