"""Linear solves and time steps (oracle; test infrastructure).

* ``dense_solve``   - direct LU of the assembled operator (tiny grids).
* ``amen_solve``    - the alternating TT solver the paper uses (AMEn; Results,
                      "Superconsistent Stabilization", Fig. 6: sweeps over the
                      cores, each with a local solve of size r_{k-1} n_k r_k).
                      The paper gives no algorithmic detail; this follows the
                      published one-site AMEn with residual enrichment
                      (Dolgov & Savostyanov 2014, cited there): Galerkin local
                      systems with left/right interface tensors, local SVD
                      truncation at tol/sqrt(d), enrichment of the new core by a
                      rank-4 approximation of the residual, which is itself
                      tracked as a TT z.  Local systems are assembled and
                      solved by LU (the paper's direct local solves: Results,
                      "Superconsistent Stabilization", local direct solves of
                      cost O((r n r)^3) dominate); above ``dense_max``
                      unknowns GMRES(40) on the same local operator is used
                      instead.  It works on any TT-matrix A and stops when
                      ``stop(x)`` (by default the relative residual
                      ||b - A x|| / ||b||) is <= tol.
* ``solve_collocation`` - AMEn for the collocation system
                      (c_mass M + c_op A) x = b.  The Galerkin local systems of
                      AMEn project the operator onto the current frames on
                      both sides, which presumes an operator from the
                      unknowns' space to itself.  The collocation operator
                      maps values at the GLL nodes (the representation grid)
                      to values at the collocation points (Overview (ii): the
                      two grids differ), so the frames are applied to the
                      equivalent node-to-node system
                          M^{-1}(c_mass M + c_op A) x = M^{-1} b,
                          M^{-1} A = sum_k I (x) .. (x) B_k (x) .. (x) I,
                          B_k = Rt_k^{-1} Lt_k,
                      a rank-2 TT-matrix of the same pattern with Rt replaced
                      by I and Lt by B_k (Rt_k is invertible: a non-zero
                      polynomial of degree N vanishing at the two boundary
                      nodes cannot vanish at N - 1 further distinct points).
                      The stopping test stays the relative residual of the
                      original collocation system.  (Galerkin AMEn on A itself
                      mixes the two grids: on the d = 6, n = 32 problem it
                      reaches only 0.48, 1.8e-2 and 1.1e-4 after sweeps 1-3,
                      while this form reaches 1.7e-11 in one sweep.)
* ``cn_step`` / ``be_step`` - eq. ttss-Crank-Nicolson and eq.
                      ttss-backward-Euler with the collocated time derivative,
                      i.e. mass matrix M = Rt (x) ... (x) Rt:
                      (M + dt/2 A) u+ = (M - dt/2 A) u;   (M + dt A) u+ = M u.

Pins (tests/test_oracle_solve.py): AMEn, on A itself and in the node-to-node
form, against the dense LU solution on tiny grids; its residual computed independently by dense algebra; the CN step
against a dense CN step and, in 1D with beta = 0 and Plain-SC, against the
closed-form amplification factor (1 - dt lam/2)/(1 + dt lam/2) of each
eigenmode of -eps D2.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse.linalg as spla

from . import tt as T
from .operator import dense, ttm_cores


def dense_solve(ops, b_tt, c_mass=0.0, c_op=1.0):
    """x = (c_mass M + c_op A)^{-1} full(b) reshaped to the grid."""
    b = T.full(b_tt)
    x = np.linalg.solve(dense(ops, c_mass, c_op), b.ravel())
    return x.reshape(b.shape)


def residual(A, b, x):
    """||b - A x||_F / ||b||_F with the accurate (orthogonalised) difference norm."""
    return T.diff_norm(b, T.matvec(A, x)) / T.norm(b)


def _local_matrix(PhiL, Ak, PhiR):
    """Dense local operator K[(a,i,b),(a',j,b')] = sum PhiL[a,p,a'] A[p,i,j,q] PhiR[b,q,b']."""
    K = np.einsum("xpy,pijq,zqw->xizyjw", PhiL, Ak, PhiR)
    ra, n, rb = K.shape[0], K.shape[1], K.shape[2]
    return K.reshape(ra * n * rb, ra * n * rb)


def _local_apply(PhiL, Ak, PhiR, X):
    return np.einsum("xpy,pijq,zqw,yjw->xiz", PhiL, Ak, PhiR, X, optimize=True)


def _phi_left(Phi, U, Ak, V):
    """Next left interface: Phi'[b,q,b'] = sum U[a,i,b] Phi[a,p,a'] A[p,i,j,q] V[a',j,b']."""
    return np.einsum("aib,apc,pijq,cjd->bqd", U, Phi, Ak, V, optimize=True)


def _phi_right(Phi, U, Ak, V):
    """Next right interface: Phi'[a,p,a'] = sum U[a,i,b] Phi[b,q,b'] A[p,i,j,q] V[a',j,b']."""
    return np.einsum("aib,bqd,pijq,cjd->apc", U, Phi, Ak, V, optimize=True)


def _vec_left(Psi, U, F):
    """Psi'[b, g'] = sum U[a,i,b] Psi[a,g] F[g,i,g']."""
    return np.einsum("aib,ag,gih->bh", U, Psi, F)


def _vec_right(Psi, U, F):
    return np.einsum("aib,bh,gih->ag", U, Psi, F)


def amen_solve(A, b, x0, tol, rmax, max_sweeps=50, kick=8, seed=0, dense_max=16000,
               verbose=False, history=None, stop=None):
    """Solve A x = b in TT format (A: TT-matrix cores, b and x0: TT cores).

    ``stop(x)`` gives the relative residual that ends the sweeps (default
    ||b - A x|| / ||b||).  Returns (x, that residual, sweeps).
    """
    if stop is None:
        def stop(v):
            return residual(A, b, v)
    d = len(b)
    ns = [c.shape[1] for c in b]
    one = np.ones((1, 1, 1))
    x = T.orth_right([c.copy() for c in x0])
    rng = np.random.default_rng(seed)
    z = T.orth_right([rng.standard_normal((1 if k == 0 else kick, ns[k], 1 if k == d - 1 else kick))
                      for k in range(d)])
    ltol = tol / math.sqrt(d)
    res = stop(x)
    sweeps = 0
    for sweep in range(max_sweeps):
        if res <= tol:
            break
        # right interfaces from the right-orthogonal x and z
        PhiR = [None] * (d + 1)
        PsiR = [None] * (d + 1)
        ZPhiR = [None] * (d + 1)
        ZPsiR = [None] * (d + 1)
        PhiR[d], ZPhiR[d] = one, one
        PsiR[d], ZPsiR[d] = np.ones((1, 1)), np.ones((1, 1))
        for k in range(d - 1, 0, -1):
            PhiR[k] = _phi_right(PhiR[k + 1], x[k], A[k], x[k])
            PsiR[k] = _vec_right(PsiR[k + 1], x[k], b[k])
            ZPhiR[k] = _phi_right(ZPhiR[k + 1], z[k], A[k], x[k])
            ZPsiR[k] = _vec_right(ZPsiR[k + 1], z[k], b[k])
        PhiL, PsiL, ZPhiL, ZPsiL = one, np.ones((1, 1)), one, np.ones((1, 1))
        for k in range(d):
            ra, n, rb = x[k].shape
            rhs = np.einsum("ag,gih,bh->aib", PsiL, b[k], PsiR[k + 1])
            N = ra * n * rb
            if N <= dense_max:
                X = np.linalg.solve(_local_matrix(PhiL, A[k], PhiR[k + 1]), rhs.ravel()).reshape(ra, n, rb)
            else:
                op = spla.LinearOperator((N, N), matvec=lambda v: _local_apply(
                    PhiL, A[k], PhiR[k + 1], v.reshape(ra, n, rb)).ravel())
                sol, _ = spla.gmres(op, rhs.ravel(), x0=x[k].ravel(), rtol=ltol, restart=40,
                                    maxiter=200)
                X = sol.reshape(ra, n, rb)
            if k == d - 1:
                x[k] = X
                break
            # truncate
            U, s, Vt = np.linalg.svd(X.reshape(ra * n, rb), full_matrices=False)
            r = T.trunc_rank(s, ltol * np.linalg.norm(s), rmax)
            U, SV = U[:, :r], s[:r, None] * Vt[:r]
            Xt = (U @ SV).reshape(ra, n, rb)
            # residual projected on (x-left) x n x (z-right): enrichment directions
            fz = np.einsum("ag,gih,bh->aib", PsiL, b[k], ZPsiR[k + 1])
            enr = fz - _local_apply(PhiL, A[k], ZPhiR[k + 1], Xt)
            # residual projected on (z-left) x n x (z-right): next z core
            fzz = np.einsum("ag,gih,bh->aib", ZPsiL, b[k], ZPsiR[k + 1])
            zr = fzz - _local_apply(ZPhiL, A[k], ZPhiR[k + 1], Xt)
            rz = z[k].shape[2]
            Uz, _, _ = np.linalg.svd(zr.reshape(-1, rz), full_matrices=False)
            zk = np.zeros((zr.shape[0], n, rz))
            zk.reshape(-1, rz)[:, :Uz.shape[1]] = Uz[:, :rz]
            z[k] = zk
            # enrich, orthogonalise, push the non-orthogonal part right
            Q, _ = np.linalg.qr(np.concatenate([U, enr.reshape(ra * n, -1)], axis=1))
            x[k] = Q.reshape(ra, n, Q.shape[1])
            x[k + 1] = np.einsum("ab,bic->aic", (Q.T @ U) @ SV, x[k + 1])
            PhiL = _phi_left(PhiL, x[k], A[k], x[k])
            PsiL = _vec_left(PsiL, x[k], b[k])
            ZPhiL = _phi_left(ZPhiL, z[k], A[k], x[k])
            ZPsiL = _vec_left(ZPsiL, z[k], b[k])
        sweeps = sweep + 1
        res = stop(x)
        if history is not None:
            history.append((res, T.ranks(x)))
        if verbose:
            print(f"sweep {sweeps}: residual {res:.3e} ranks {T.ranks(x)}")
        x = T.orth_right(x)
    return x, res, sweeps


class _NodeOp:
    """The 1D pieces of M^{-1} A for one dimension: Rt -> I, Lt -> Rt^{-1} Lt."""

    def __init__(self, o):
        m = o.Rt.shape[0]
        self.Rt = np.eye(m)
        self.Lt = np.linalg.solve(o.Rt, o.Lt)
        self.Rinv = np.linalg.inv(o.Rt)


def solve_collocation(ops, b, x0, tol, rmax, c_mass=0.0, c_op=1.0, max_sweeps=50, **kw):
    """(c_mass M + c_op A) x = b by AMEn on M^{-1}(c_mass M + c_op A) x = M^{-1} b,
    stopping on the residual of the original system.  ``ops`` are the 1D
    pieces (Rt, Lt per dimension, in TT order).  Returns (x, residual, sweeps)."""
    nops = [_NodeOp(o) for o in ops]
    Ak = ttm_cores(nops, c_mass, c_op)
    bk = [np.einsum("ij,ajb->aib", o.Rinv, c) for o, c in zip(nops, b)]
    A = ttm_cores(ops, c_mass, c_op)
    return amen_solve(Ak, bk, x0, tol, rmax, max_sweeps=max_sweeps, stop=lambda v: residual(A, b, v), **kw)


def cn_rhs(ops, u, dt, tol, rmax):
    """(M - dt/2 A) u, rounded."""
    return T.round_tt(T.matvec(ttm_cores(ops, 1.0, -0.5 * dt), u), tol, rmax)


def cn_step(ops, u, dt, tol, rmax, max_sweeps=20):
    """One Crank-Nicolson step (eq. ttss-Crank-Nicolson, mass matrix M = (x) Rt)."""
    rhs = cn_rhs(ops, u, dt, tol, rmax)
    return solve_collocation(ops, rhs, u, tol, rmax, 1.0, 0.5 * dt, max_sweeps)


def be_step(ops, u, dt, tol, rmax, max_sweeps=20):
    """One backward-Euler step (eq. ttss-backward-Euler): (M + dt A) u+ = M u."""
    rhs = T.round_tt(T.matvec(ttm_cores(ops, 1.0, 0.0), u), tol, rmax)
    return solve_collocation(ops, rhs, u, tol, rmax, 1.0, dt, max_sweeps)
