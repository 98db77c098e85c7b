"""Pins for the oracle's tensor-train arithmetic (Methods, "Tensor Train representation")."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import tt as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense_low_rank(shape, rank, rng):
    """Sum of `rank` random separable terms (TT ranks <= rank)."""
    A = 0.0
    for _ in range(rank):
        t = rng.standard_normal(shape[0])
        for n in shape[1:]:
            t = np.multiply.outer(t, rng.standard_normal(n))
        A = A + t
    return A


def test_full_matches_elementwise_slice_products():
    # eq. TT-format:elementwise / eq. TT-format:slice, by brute force.
    x = W.random_tt(4, (3, 4, 2, 3), [1, 2, 3, 2, 1], seed=5)
    F = T.full(x)
    for idx in itertools.product(*[range(s) for s in F.shape]):
        s = 0.0
        for a in itertools.product(range(2), range(3), range(2)):
            s += x[0][0, idx[0], a[0]] * x[1][a[0], idx[1], a[1]] * x[2][a[1], idx[2], a[2]] * x[3][a[2], idx[3], 0]
        assert abs(F[idx] - s) < 1e-13
        assert abs(T.element(x, idx) - s) < 1e-13


def test_fig2_entry_is_product_of_slices():
    g = json.load(open(os.path.join(GOLDEN, "paper_printed_numbers.json")))["fig2_entry"]
    idx = [i - 1 for i in g["index_one_based"]]
    x = W.random_tt(6, 8, [1, 3, 2, 4, 2, 3, 1], seed=11)
    m = np.eye(1)
    for k, i in enumerate(idx):
        m = m @ x[k][:, i, :]
    assert abs(T.full(x)[tuple(idx)] - m[0, 0]) < 1e-13


def test_storage_and_compression_printed_numbers():
    g = json.load(open(os.path.join(GOLDEN, "paper_printed_numbers.json")))
    s = g["storage_remark"]
    assert s["d"] * s["n"] * s["r"] ** 2 == s["printed_tt_storage"]
    assert float(s["n"]) ** s["d"] == s["printed_full_storage"]
    c = g["compression_E1"]
    ratio = c["d"] * c["r"] ** 2 * c["n"] / float(c["n"]) ** c["d"]
    assert 0.1 * c["printed_order"] < ratio < 10 * c["printed_order"]
    # with exact boundary ranks r_0 = r_d = 1 the TT storage is below the estimate
    ranks = [1] + [c["r"]] * (c["d"] - 1) + [1]
    exact = sum(ranks[k] * c["n"] * ranks[k + 1] for k in range(c["d"]))
    assert exact <= c["d"] * c["r"] ** 2 * c["n"]


@pytest.mark.parametrize("shape,rank", [((4, 5, 6), 2), ((3, 4, 3, 5), 3), ((6, 6, 6, 6), 1)])
def test_tt_svd_exact_with_unfolding_ranks(shape, rank):
    rng = np.random.default_rng(sum(shape) + rank)
    A = _dense_low_rank(shape, rank, rng)
    x = T.tt_svd(A, 1e-14)
    for k in range(1, len(shape)):
        unf = A.reshape(int(np.prod(shape[:k])), -1)
        assert T.ranks(x)[k] == np.linalg.matrix_rank(unf, tol=1e-10 * np.linalg.norm(A))
    assert np.linalg.norm(T.full(x) - A) < 1e-13 * np.linalg.norm(A)


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-4])
def test_tt_svd_error_bound(eps):
    rng = np.random.default_rng(3)
    for _ in range(5):
        A = rng.standard_normal((5, 6, 4, 5)) + _dense_low_rank((5, 6, 4, 5), 2, rng) * 3
        x = T.tt_svd(A, eps)
        err = np.linalg.norm(T.full(x) - A)
        assert err <= eps * math.sqrt(3) * np.linalg.norm(A) * (1 + 1e-12)


@pytest.mark.parametrize("eps", [0.3, 1e-1, 1e-3, 1e-6])
def test_rounding_error_bound_and_idempotence(eps):
    for seed in range(4):
        x = W.random_tt(5, (4, 5, 3, 6, 4), [1, 4, 7, 6, 5, 1], seed=seed)
        A = T.full(x)
        y = T.round_tt(x, eps)
        assert np.linalg.norm(T.full(y) - A) <= eps * np.linalg.norm(A) * (1 + 1e-12)
        # a rounded TT already has minimal ranks: rounding it again at a tiny
        # tolerance keeps its ranks and its content
        z = T.round_tt(y, 1e-13)
        assert T.ranks(z) == T.ranks(y)
        assert np.linalg.norm(T.full(z) - T.full(y)) <= 1e-12 * np.linalg.norm(A)


def test_rounding_ranks_bounded_by_unfolding_ranks():
    rng = np.random.default_rng(8)
    A = _dense_low_rank((4, 5, 4, 5), 2, rng)
    x = T.tt_svd(A, 1e-15)
    x2 = T.add(x, x)  # rank doubles, content 2A
    y = T.round_tt(x2, 1e-12)
    assert max(T.ranks(y)) <= 2
    assert np.linalg.norm(T.full(y) - 2 * A) < 1e-11 * np.linalg.norm(A)


def test_duplicated_rank1_rounds_back_to_rank1():
    rng = np.random.default_rng(9)
    x = [rng.standard_normal((1, n, 1)) for n in (5, 6, 7, 4)]
    y = T.round_tt(T.add(x, T.scale(x, 0.5)), 1e-12)
    assert T.ranks(y) == [1, 1, 1, 1, 1]
    assert np.linalg.norm(T.full(y) - 1.5 * T.full(x)) < 1e-12 * np.linalg.norm(T.full(x))


def test_rounding_of_a_cancelling_pair_against_dense():
    """t1 - t1 + 1e-9 t2 + t3 on a grid small enough to hold densely: at
    tolerance 0 the rounding reproduces the dense tensor to roundoff, and at
    a tolerance above the 1e-9 part it keeps rank <= r and lands within the
    error bound of t3 + 1e-9 t2 (the exactly cancelling pair carries
    nothing)."""
    d, m, r = 4, 6, 2
    t1 = W.random_tt(d, m, [1] + [r] * (d - 1) + [1], seed=41)
    t2 = W.random_tt(d, m, [1] + [r] * (d - 1) + [1], seed=42)
    t3 = W.random_tt(d, m, [1] + [r] * (d - 1) + [1], seed=43)
    x = T.add(T.add(T.add(t1, T.scale(t1, -1.0)), T.scale(t2, 1e-9)), t3)
    x[0] = x[0] / 1e3
    x[-1] = x[-1] * 1e3
    dense = T.full(t3) + 1e-9 * T.full(t2)
    assert np.linalg.norm(T.full(x) - dense) <= 1e-14 * np.linalg.norm(dense)
    y0 = T.round_tt(x, 0.0)
    assert np.linalg.norm(T.full(y0) - dense) <= 1e-13 * np.linalg.norm(dense)
    y = T.round_tt(x, 1e-6)
    assert max(T.ranks(y)) <= r
    assert np.linalg.norm(T.full(y) - dense) <= 1e-6 * np.linalg.norm(dense)


def test_add_scale_dot_norm_against_dense():
    x = W.random_tt(4, (3, 4, 5, 3), [1, 2, 3, 2, 1], seed=1)
    y = W.random_tt(4, (3, 4, 5, 3), [1, 3, 2, 4, 1], seed=2)
    X, Y = T.full(x), T.full(y)
    assert np.allclose(T.full(T.add(x, y)), X + Y, atol=1e-13)
    assert np.allclose(T.full(T.scale(x, -2.5)), -2.5 * X, atol=1e-13)
    assert abs(T.dot(x, y) - np.sum(X * Y)) < 1e-12
    assert abs(T.norm(x) - np.linalg.norm(X)) < 1e-12
    assert abs(T.diff_norm(x, y) - np.linalg.norm(X - Y)) < 1e-12


def test_diff_norm_sees_tiny_differences():
    # the orthogonalised difference resolves ||x - y|| = 1e-13 ||x||, which
    # sqrt(<x,x> - 2<x,y> + <y,y>) cannot.
    x = W.random_tt(5, 6, [1, 3, 4, 4, 3, 1], seed=4)
    dx = W.random_tt(5, 6, [1, 2, 2, 2, 2, 1], seed=5)
    nx = T.norm(x)
    delta = 1e-13 * nx / T.norm(dx)
    y = T.add(x, T.scale(dx, delta))
    exact = np.linalg.norm(T.full(y) - T.full(x))
    assert abs(T.diff_norm(y, x) - exact) < 1e-3 * exact


def test_orthogonalisation_properties():
    x = W.random_tt(4, (5, 4, 6, 3), [1, 3, 4, 3, 1], seed=6)
    r = T.orth_right(x)
    for c in r[1:]:
        m = c.reshape(c.shape[0], -1)
        assert np.allclose(m @ m.T, np.eye(m.shape[0]), atol=1e-13)
    l = T.orth_left(x)
    for c in l[:-1]:
        m = c.reshape(-1, c.shape[2])
        assert np.allclose(m.T @ m, np.eye(m.shape[1]), atol=1e-13)
    assert np.allclose(T.full(r), T.full(x), atol=1e-13)
    assert np.allclose(T.full(l), T.full(x), atol=1e-13)


def test_matvec_against_dense():
    rng = np.random.default_rng(12)
    A = []
    ns = (3, 4, 3)
    Rk = [1, 2, 3, 1]
    for k, n in enumerate(ns):
        A.append(rng.standard_normal((Rk[k], n, n, Rk[k + 1])))
    x = W.random_tt(3, ns, [1, 2, 2, 1], seed=3)
    y = T.matvec(A, x)
    assert np.allclose(T.full(y).ravel(), T.ttm_full(A) @ T.full(x).ravel(), atol=1e-12)
