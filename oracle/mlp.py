"""Learned warm start: an MLP from problem parameters to TT cores (oracle;
test infrastructure -- only tests/, the smoke check and bench.py's CPU
baseline may import it).

The paper's solver accepts any initial guess and always runs to the same
residual tolerance (Results, AMEn initial guess); a better guess only saves
sweeps.  This module is the plain FP64 reference of the network that
supplies that guess:

    h1 = relu(W1 p + b1),  h2 = relu(W2 h1 + b2),  y = W3 h2 + b3,

with y read as raw TT cores Y_k (core 0 of shape (1, m_1, r), middle cores
(r, m_k, r), last core (r, m_d, 1), each row-major, concatenated in order)
followed by one log-scale sigma.  The tensor X(p) has the cores
X_k = Y_k / ||Y_k||_F, with core 0 also multiplied by exp(sigma): each core
enters through its direction only and the overall size through sigma.  (The
loss is a polynomial of degree 2d in raw cores; normalised cores keep it well
conditioned, and the alternating solver that consumes X(p) does not depend on
the scale of its initial guess anyway.)  The loss of one sample with target
tensor U (a TT of any ranks) is the gauge-invariant relative error

    L = ||X - U||_F^2 / ||U||_F^2 = (<X,X> - 2 <X,U> + <U,U>) / <U,U>,

evaluated with TT inner products, and averaged over the batch.  Gradients
are by hand: dL/dX_k from the left and right environments of <X,X> and
<X,U>, then through the normalisation (dL/dY = (g - <g, Yhat> Yhat) / ||Y||
with g = dL/dYhat, and dL/dsigma = <dL/dX_0, X_0>), then ordinary
backpropagation through the three layers (relu'(0) = 0).
Adam follows Kingma & Ba with bias correction (beta1 0.9, beta2 0.999,
epsilon 1e-8).

Weights are row-major (out x in).  Pins (tests/test_oracle_mlp.py): central
finite differences of the loss in FP64 on a small network, loss against the
dense tensors, gauge invariance, zero loss at X = U, invariance under scaling
of a raw core, the exp(sigma) norm law, and Adam's first steps in closed
form.
"""
from __future__ import annotations

import numpy as np

from . import tt as OT


def core_dim(d, m, r):
    """Number of raw core entries for d cores of mode sizes m (list) and rank r."""
    if d == 1:
        return m[0]
    return m[0] * r + sum(r * m[k] * r for k in range(1, d - 1)) + r * m[d - 1]


def out_dim(d, m, r):
    """Length of y: the raw cores and the log-scale."""
    return core_dim(d, m, r) + 1


def raw_cores(y, d, m, r):
    """The raw cores Y_k of y (see module docstring)."""
    cores, o = [], 0
    for k in range(d):
        a = 1 if k == 0 else r
        b = 1 if k == d - 1 else r
        n = a * m[k] * b
        cores.append(np.asarray(y[o:o + n]).reshape(a, m[k], b))
        o += n
    assert o + 1 == len(y)
    return cores


def split_cores(y, d, m, r):
    """TT cores of X(p): normalised raw cores, core 0 scaled by exp(sigma)."""
    cores = [c / np.linalg.norm(c) for c in raw_cores(y, d, m, r)]
    cores[0] = cores[0] * np.exp(y[-1])
    return cores


def init_params(in_dim, hidden, odim, seed):
    """He-style normal initialisation (any initialisation serves the pins)."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((hidden, in_dim)) * np.sqrt(2.0 / in_dim), "b1": np.zeros(hidden),
        "W2": rng.standard_normal((hidden, hidden)) * np.sqrt(2.0 / hidden), "b2": np.zeros(hidden),
        "W3": rng.standard_normal((odim, hidden)) * np.sqrt(1.0 / hidden), "b3": np.zeros(odim),
    }


def forward(params, P):
    """Batch forward pass; P is (batch, in_dim).  Returns y and the hidden states."""
    z1 = P @ params["W1"].T + params["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ params["W3"].T + params["b3"]
    return y, (z1, h1, z2, h2)


def _left_envs(x, u):
    """E[k] = contraction of cores 0..k-1 of x and u: shape (r_x[k], r_u[k])."""
    E = [np.ones((1, 1))]
    for a, b in zip(x, u):
        E.append(np.einsum("ac,aib,cid->bd", E[-1], a, b))
    return E


def _right_envs(x, u):
    """F[k] = contraction of cores k..d-1: shape (r_x[k], r_u[k]); F[d] = 1."""
    d = len(x)
    F = [None] * (d + 1)
    F[d] = np.ones((1, 1))
    for k in range(d - 1, -1, -1):
        F[k] = np.einsum("aib,cid,bd->ac", x[k], u[k], F[k + 1])
    return F


def tt_loss(x, u):
    """||X - U||^2 / ||U||^2 through TT inner products."""
    uu = OT.dot(u, u)
    return (OT.dot(x, x) - 2.0 * OT.dot(x, u) + uu) / uu


def tt_loss_grad(x, u):
    """Loss of one sample and dL/dX_k for every core.

    d<X,X>/dX_k[a,i,b] = 2 sum EL[a,a'] X_k[a',i,b'] ER[b,b'] (EL, ER: left and
    right environments of <X,X>); d<X,U>/dX_k[a,i,b] = sum FL[a,c] U_k[c,i,c']
    FR[b,c'] (environments of <X,U>).
    """
    uu = OT.dot(u, u)
    Lxx, Rxx = _left_envs(x, x), _right_envs(x, x)
    Lxu, Rxu = _left_envs(x, u), _right_envs(x, u)
    xx = float(Lxx[-1][0, 0])
    xu = float(Lxu[-1][0, 0])
    loss = (xx - 2.0 * xu + uu) / uu
    grads = []
    for k in range(len(x)):
        gxx = 2.0 * np.einsum("ae,eif,bf->aib", Lxx[k], x[k], Rxx[k + 1])
        gxu = np.einsum("ac,cid,bd->aib", Lxu[k], u[k], Rxu[k + 1])
        grads.append((gxx - 2.0 * gxu) / uu)
    return loss, grads


def loss_and_grads(params, P, targets, d, m, r):
    """Mean loss over the batch and its gradients with respect to every parameter."""
    y, (z1, h1, z2, h2) = forward(params, P)
    B = P.shape[0]
    dy = np.zeros_like(y)
    total = 0.0
    for s in range(B):
        raw = raw_cores(y[s], d, m, r)
        x = split_cores(y[s], d, m, r)
        loss, g = tt_loss_grad(x, targets[s])
        total += loss
        sig = y[s, -1]
        parts = []
        for k in range(d):
            nk = np.linalg.norm(raw[k])
            yhat = raw[k] / nk
            gh = g[k] * np.exp(sig) if k == 0 else g[k]  # dL/dYhat_k
            parts.append(((gh - np.sum(gh * yhat) * yhat) / nk).ravel())
        parts.append(np.array([np.sum(g[0] * x[0])]))    # dL/dsigma
        dy[s] = np.concatenate(parts) / B
    grads = {}
    grads["W3"] = dy.T @ h2
    grads["b3"] = dy.sum(axis=0)
    dh2 = dy @ params["W3"]
    dz2 = dh2 * (z2 > 0)
    grads["W2"] = dz2.T @ h1
    grads["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ params["W2"]
    dz1 = dh1 * (z1 > 0)
    grads["W1"] = dz1.T @ P
    grads["b1"] = dz1.sum(axis=0)
    return total / B, grads


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state holds t and the moment estimates."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m *= beta1
        m += (1.0 - beta1) * grads[k]
        v *= beta2
        v += (1.0 - beta2) * grads[k] ** 2
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        params[k] -= lr * mhat / (np.sqrt(vhat) + eps)
    return params
