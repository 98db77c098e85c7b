"""Pins of the warm-start network oracle (oracle/mlp.py).

Gradients against central finite differences in FP64 on a 15 -> 8 -> 8 ->
(d = 3, m = 4, rank 2 TT) network; the TT loss against dense tensors; gauge
invariance; zero loss at the target; Adam's first two steps in closed form.
"""
import numpy as np
import pytest

from oracle import mlp as M
from oracle import tt as OT
import workloads as W

D, MM, R = 3, [4, 5, 3], 2


def _setup(seed=0, batch=3):
    rng = np.random.default_rng(seed)
    odim = M.out_dim(D, MM, R)
    params = M.init_params(15, 8, odim, seed)
    for k in ("b1", "b2", "b3"):
        params[k] = 0.1 * rng.standard_normal(params[k].shape)
    P = rng.standard_normal((batch, 15))
    targets = [W.random_tt(D, MM, [1, 3, 2, 1], seed=seed * 10 + s) for s in range(batch)]
    return params, P, targets


def test_out_dim_and_split():
    odim = M.out_dim(D, MM, R)
    assert odim == 4 * 2 + 2 * 5 * 2 + 2 * 3 + 1
    y = np.arange(odim, dtype=float) / odim
    raw = M.raw_cores(y, D, MM, R)
    assert [c.shape for c in raw] == [(1, 4, 2), (2, 5, 2), (2, 3, 1)]
    assert raw[1][0, 0, 0] == y[8] and raw[2][1, 2, 0] == y[odim - 2]
    cores = M.split_cores(y, D, MM, R)
    # unit-norm cores, the first scaled by exp(sigma)
    assert abs(np.linalg.norm(cores[0]) - np.exp(y[-1])) <= 1e-12 * np.exp(y[-1])
    assert all(abs(np.linalg.norm(c) - 1.0) <= 1e-14 for c in cores[1:])


def test_loss_ignores_the_scale_of_each_raw_core():
    params, P, targets = _setup()
    y, _ = M.forward(params, P)
    x0 = M.split_cores(y[0], D, MM, R)
    # scaling one raw core leaves X (and so the loss) unchanged
    y2 = y[0].copy()
    y2[8:28] *= 3.7
    x2 = M.split_cores(y2, D, MM, R)
    assert all(np.allclose(a, b, rtol=1e-14, atol=0) for a, b in zip(x0, x2))
    # sigma moves the norm of X exactly by exp(sigma)
    y3 = y[0].copy()
    y3[-1] += 0.5
    assert abs(OT.norm(M.split_cores(y3, D, MM, R)) / OT.norm(x0) - np.exp(0.5)) <= 1e-13


def test_tt_loss_matches_dense():
    x = W.random_tt(D, MM, [1, 2, 2, 1], seed=1)
    u = W.random_tt(D, MM, [1, 3, 2, 1], seed=2)
    dense = np.sum((OT.full(x) - OT.full(u)) ** 2) / np.sum(OT.full(u) ** 2)
    assert abs(M.tt_loss(x, u) - dense) <= 1e-13 * dense
    loss, _ = M.tt_loss_grad(x, u)
    assert abs(loss - dense) <= 1e-13 * dense


def test_loss_zero_at_target_in_another_gauge():
    u = W.random_tt(D, MM, [1, 2, 2, 1], seed=3)
    G = np.array([[2.0, 1.0], [0.5, 1.5]])
    x = [np.einsum("aib,bc->aic", u[0], G), np.einsum("ab,bic->aic", np.linalg.inv(G), u[1]), u[2].copy()]
    assert abs(M.tt_loss(x, u)) <= 1e-13
    _, g = M.tt_loss_grad(x, u)
    assert max(np.max(np.abs(gk)) for gk in g) <= 1e-12


def test_core_gradient_is_gauge_covariant():
    # the loss is gauge invariant, so at a gauge transform the gradient of
    # core 0 transforms with G^{-T}: <grad_0, dX_0> is unchanged for dX = E G
    x = W.random_tt(D, MM, [1, 2, 2, 1], seed=4)
    u = W.random_tt(D, MM, [1, 3, 2, 1], seed=5)
    G = np.array([[1.0, 0.3], [-0.2, 0.8]])
    xg = [np.einsum("aib,bc->aic", x[0], G), np.einsum("ab,bic->aic", np.linalg.inv(G), x[1]), x[2]]
    _, g = M.tt_loss_grad(x, u)
    _, gg = M.tt_loss_grad(xg, u)
    assert np.allclose(np.einsum("aic,bc->aib", gg[0], G), g[0], rtol=1e-11, atol=1e-13)


def test_gradients_match_central_differences():
    params, P, targets = _setup()
    _, grads = M.loss_and_grads(params, P, targets, D, MM, R)
    h = 1e-6
    rng = np.random.default_rng(7)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = params[k].ravel()
        idxs = rng.choice(flat.size, size=min(flat.size, 12), replace=False)
        for i in idxs:
            old = flat[i]
            flat[i] = old + h
            lp, _ = M.loss_and_grads(params, P, targets, D, MM, R)
            flat[i] = old - h
            lm, _ = M.loss_and_grads(params, P, targets, D, MM, R)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = grads[k].ravel()[i]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)), (k, i, fd, an)


def test_core_gradient_matches_central_differences():
    x = W.random_tt(D, MM, [1, 2, 2, 1], seed=8)
    u = W.random_tt(D, MM, [1, 3, 2, 1], seed=9)
    _, g = M.tt_loss_grad(x, u)
    h = 1e-6
    for k in range(D):
        for idx in np.ndindex(*x[k].shape):
            old = x[k][idx]
            x[k][idx] = old + h
            lp = M.tt_loss(x, u)
            x[k][idx] = old - h
            lm = M.tt_loss(x, u)
            x[k][idx] = old
            assert abs((lp - lm) / (2 * h) - g[k][idx]) <= 1e-6 * max(1e-3, abs(g[k][idx]))


def test_relu_derivative_at_zero_is_zero():
    params, P, targets = _setup(batch=1)
    # force every first-layer pre-activation to exactly zero
    params["W1"][:] = 0.0
    params["b1"][:] = 0.0
    _, grads = M.loss_and_grads(params, P, targets[:1], D, MM, R)
    assert np.all(grads["W1"] == 0) and np.all(grads["b1"] == 0) and np.all(grads["W2"] == 0)


def test_adam_first_steps_closed_form():
    lr = 1e-2
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -0.1, 0.0])}
    st = {}
    M.adam_step(p, g, st, lr)
    # after one step the bias-corrected moments are g and g^2
    exp1 = np.array([1.0, -2.0, 0.5]) - lr * g["w"] / (np.abs(g["w"]) + 1e-8)
    assert np.allclose(p["w"], exp1, rtol=0, atol=1e-15)
    M.adam_step(p, g, st, lr)
    # a constant gradient keeps mhat = g and vhat = g^2 at every step
    exp2 = exp1 - lr * g["w"] / (np.abs(g["w"]) + 1e-8)
    assert np.allclose(p["w"], exp2, rtol=0, atol=1e-15)
    assert st["t"] == 2
