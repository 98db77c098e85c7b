"""Tensor-train format and its arithmetic (oracle; test infrastructure).

Methods, "Tensor Train representation": a TT tensor is a list of cores
G_k of shape (r_{k-1}, n_k, r_k) with r_0 = r_d = 1 (eq. TT-format:elementwise);
a TT-matrix has cores L_k of shape (R_{k-1}, n_k, n_k, R_k) indexed
L_k(alpha, i, j, beta) (eq. tt-matrix-format).  TT-SVD builds a TT by
sequential truncated SVDs of the unfoldings with error at most
eps sqrt(d-1) ||A||_F; rounding recompresses with error at most eps ||A||_F.

Pins (tests/test_oracle_tt.py): full() against the elementwise slice-product
definition (eq. TT-format:slice) by brute force; TT-SVD exact with the
unfolding ranks (Theorem 2.1 of the cited TT paper, restated in Methods) and
rank 1 for separable data; both error bounds on random tensors; rounding
idempotence; add/dot/matvec against dense numpy on tiny cases.
"""
from __future__ import annotations

import math

import numpy as np


def ranks(cores):
    return [cores[0].shape[0]] + [c.shape[2] for c in cores]


def full(cores):
    """Dense tensor of shape (n_1, ..., n_d)."""
    shape = [c.shape[1] for c in cores]
    t = cores[0].reshape(cores[0].shape[1], cores[0].shape[2])
    for c in cores[1:]:
        t = t @ c.reshape(c.shape[0], -1)
        t = t.reshape(-1, c.shape[2])
    return t.reshape(shape)


def element(cores, idx):
    """A(i_1..i_d) = G_1(i_1) G_2(i_2) ... G_d(i_d) (slice form)."""
    m = np.ones((1, 1))
    for c, i in zip(cores, idx):
        m = m @ c[:, i, :]
    return float(m[0, 0])


def trunc_rank(s, delta, rmax=None):
    """Smallest r >= 1 with sqrt(sum_{j >= r} s_j^2) <= delta, then capped at rmax.

    Ties (tail equal to delta within 1e-14 relative) keep the larger rank.
    """
    tail = np.sqrt(np.cumsum((s * s)[::-1]))[::-1]  # tail[j] = ||s[j:]||
    r = len(s)
    for j in range(1, len(s)):
        if tail[j] < delta * (1.0 - 1e-14):
            r = j
            break
    if rmax is not None:
        r = min(r, rmax)
    return max(r, 1)


def tt_svd(A, eps, rmax=None):
    """TT-SVD with per-unfolding threshold delta = eps ||A||_F / sqrt(d-1)."""
    A = np.asarray(A, dtype=np.float64)
    d, n = A.ndim, A.shape
    delta = eps * np.linalg.norm(A) / math.sqrt(max(d - 1, 1))
    cores, r, C = [], 1, A
    for k in range(d - 1):
        C = C.reshape(r * n[k], -1)
        U, s, Vt = np.linalg.svd(C, full_matrices=False)
        rk = trunc_rank(s, delta, rmax)
        cores.append(U[:, :rk].reshape(r, n[k], rk))
        C = s[:rk, None] * Vt[:rk]
        r = rk
    cores.append(C.reshape(r, n[-1], 1))
    return cores


def add(x, y):
    """x + y with block-diagonal cores (ranks add)."""
    d = len(x)
    if d == 1:
        return [x[0] + y[0]]
    out = []
    for k, (a, b) in enumerate(zip(x, y)):
        ra, n, sa = a.shape
        rb, _, sb = b.shape
        if k == 0:
            out.append(np.concatenate([a, b], axis=2))
        elif k == d - 1:
            out.append(np.concatenate([a, b], axis=0))
        else:
            c = np.zeros((ra + rb, n, sa + sb))
            c[:ra, :, :sa] = a
            c[ra:, :, sa:] = b
            out.append(c)
    return out


def scale(x, a):
    return [x[0] * a] + [c.copy() for c in x[1:]]


def dot(x, y):
    """<x, y> by left-to-right contraction of the interface matrices."""
    phi = np.ones((1, 1))
    for a, b in zip(x, y):
        phi = np.einsum("pq,pib,qic->bc", phi, a, b)
    return float(phi[0, 0])


def orth_right(x):
    """Right-to-left orthogonalisation: cores 2..d get orthonormal rows (r_{k-1} x n r_k)."""
    x = [c.copy() for c in x]
    for k in range(len(x) - 1, 0, -1):
        r0, n, r1 = x[k].shape
        Q, Rf = np.linalg.qr(x[k].reshape(r0, n * r1).T)   # G^T = Q R  ->  G = R^T Q^T
        rn = Q.shape[1]
        x[k] = Q.T.reshape(rn, n, r1)
        x[k - 1] = np.einsum("aib,cb->aic", x[k - 1], Rf)
    return x


def orth_left(x):
    """Left-to-right orthogonalisation: cores 1..d-1 get orthonormal columns."""
    x = [c.copy() for c in x]
    for k in range(len(x) - 1):
        r0, n, r1 = x[k].shape
        Q, Rf = np.linalg.qr(x[k].reshape(r0 * n, r1))
        rn = Q.shape[1]
        x[k] = Q.reshape(r0, n, rn)
        x[k + 1] = np.einsum("ab,bic->aic", Rf, x[k + 1])
    return x


def norm(x):
    """||x||_F via orthogonalisation (no cancellation): the norm of the first core."""
    return float(np.linalg.norm(orth_right(x)[0]))


def diff_norm(x, y):
    """||x - y||_F, formed as the TT x + (-y) and orthogonalised."""
    return norm(add(x, scale(y, -1.0)))


def round_tt(x, eps, rmax=None):
    """TT rounding: right-to-left QR, then left-to-right truncated SVD.

    Threshold per unfolding delta = eps ||x||_F / sqrt(d-1); the cap rmax is
    applied after delta.  Guarantees ||x - round(x)||_F <= eps ||x||_F when no
    cap binds.
    """
    d = len(x)
    x = orth_right(x)
    if d == 1:
        return x
    nrm = np.linalg.norm(x[0])
    delta = eps * nrm / math.sqrt(d - 1)
    for k in range(d - 1):
        r0, n, r1 = x[k].shape
        U, s, Vt = np.linalg.svd(x[k].reshape(r0 * n, r1), full_matrices=False)
        rk = trunc_rank(s, delta, rmax)
        x[k] = U[:, :rk].reshape(r0, n, rk)
        x[k + 1] = np.einsum("ab,bic->aic", s[:rk, None] * Vt[:rk], x[k + 1])
    return x


def matvec(A, x):
    """TT-matrix by TT: Y_k[(alpha,a), i, (beta,b)] = sum_j A_k[alpha,i,j,beta] X_k[a,j,b]."""
    out = []
    for L, X in zip(A, x):
        Ra, n, _, Rb = L.shape
        ra, _, rb = X.shape
        Y = np.einsum("pijq,ajb->paiqb", L, X)
        out.append(Y.reshape(Ra * ra, n, Rb * rb))
    return out


def ttm_full(A):
    """Dense matrix of a TT-matrix (tiny cases): rows (i_1..i_d), cols (j_1..j_d)."""
    M = A[0][0]  # (n, n, R1)
    M = M[None]
    for L in A[1:]:
        M = np.einsum("xijp,pklq->xikjlq", M, L)
        s = M.shape
        M = M.reshape(s[0], s[1] * s[2], s[3] * s[4], s[5])
    return M[0, :, :, 0]
