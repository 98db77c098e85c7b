"""Host-side input preparation for the library (no method arithmetic on the device path).

Samples a workload's analytic factors at the nodes the library reports
(t2s2_op_nodes) and lays them out as TT cores:

* ``source_cores``: b = -eps Laplace u* + beta . grad u* on the collocation
  grid, built exactly from separable terms (the paper derives sources from
  analytic solutions, Results "Global Accuracy"); one rank-2 block per term.
* ``solution_cores``: u* (or an initial condition) on the interior GLL grid,
  one rank-1 block per term; ``full_solution_cores`` the same on every GLL
  node (Dirichlet data).
* ``spacetime_*``: the same for the unified space-time form (time as one
  more collocated dimension, first): the source before the initial
  condition is lifted, and the initial condition itself.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def _block_tt(blocks):
    """Concatenate per-term TT blocks (lists of cores) along the ranks."""
    d = len(blocks[0])
    if d == 1:
        return [sum(b[0] for b in blocks)]
    out = []
    for k in range(d):
        if k == 0:
            out.append(np.concatenate([b[0] for b in blocks], axis=2))
        elif k == d - 1:
            out.append(np.concatenate([b[k] for b in blocks], axis=0))
        else:
            ra = sum(b[k].shape[0] for b in blocks)
            rb = sum(b[k].shape[2] for b in blocks)
            c = np.zeros((ra, blocks[0][k].shape[1], rb))
            a0 = b0 = 0
            for b in blocks:
                c[a0:a0 + b[k].shape[0], :, b0:b0 + b[k].shape[2]] = b[k]
                a0 += b[k].shape[0]
                b0 += b[k].shape[2]
            out.append(c)
    return out


def source_cores(problem, op):
    d, eps = problem.d, problem.eps
    blocks = []
    for t in problem.terms:
        cores = []
        for k in range(d):
            _, eta = op.nodes(k)
            f = t.factors[k]
            p = f(eta)
            l = float(problem.beta[k]) * f(eta, 1) - eps * f(eta, 2)
            n = len(eta)
            if d == 1:
                c = l.reshape(1, n, 1)
            elif k == 0:
                c = np.stack([l, p], axis=1).reshape(1, n, 2)
            elif k == d - 1:
                c = np.stack([p, l], axis=0).reshape(2, n, 1)
            else:
                c = np.zeros((2, n, 2))
                c[0, :, 0] = p
                c[1, :, 0] = l
                c[1, :, 1] = p
            cores.append(c)
        cores[0] = cores[0] * t.coef
        blocks.append(cores)
    return _block_tt(blocks)


def varcoef_source_cores(vp, op):
    """b = -eps Laplace u* + beta . grad u* + rho u* on the collocation grid
    for a workloads.VarCoefProblem: per term and dimension the factor
    beta_k(eta) phi' - eps phi'' + (rho_k(eta) [+ rho0 for k = 0]) phi, and
    with a product reaction one more rank-1 block per term."""
    problem = vp.problem
    d, eps = problem.d, problem.eps
    blocks = []
    for t in problem.terms:
        cores = []
        for k in range(d):
            _, eta = op.nodes(k)
            f = t.factors[k]
            p = f(eta)
            rho = vp.rho_fn(k)(eta) + (vp.rho0 if k == 0 else 0.0)
            l = vp.beta_fn(k)(eta) * f(eta, 1) - eps * f(eta, 2) + rho * p
            n = len(eta)
            if d == 1:
                c = l.reshape(1, n, 1)
            elif k == 0:
                c = np.stack([l, p], axis=1).reshape(1, n, 2)
            elif k == d - 1:
                c = np.stack([p, l], axis=0).reshape(2, n, 1)
            else:
                c = np.zeros((2, n, 2))
                c[0, :, 0] = p
                c[1, :, 0] = l
                c[1, :, 1] = p
            cores.append(c)
        cores[0] = cores[0] * t.coef
        blocks.append(cores)
        if vp.prod:
            # the product reaction of this term, prod_k pi_k(eta) phi_k(eta)
            prod = []
            for k in range(d):
                _, eta = op.nodes(k)
                prod.append((vp.prod_fn(k)(eta) * t.factors[k](eta)).reshape(1, -1, 1))
            prod[0] = prod[0] * t.coef
            blocks.append(prod)
    return _block_tt(blocks)


def build_operator_var(vp, stream=None):
    """The library operator of a workloads.VarCoefProblem."""
    from . import t2s2_build_operator_var
    p = vp.problem
    return t2s2_build_operator_var(p.d, p.n, p.beta, p.eps, [vp.beta_fn(k) for k in range(p.d)],
                                   [vp.rho_fn(k) for k in range(p.d)], vp.rho0, p.plain_sc, stream,
                                   [vp.prod_fn(k) for k in range(p.d)] if vp.prod else None)


def solution_cores(problem, op):
    blocks = []
    for t in problem.terms:
        cores = []
        for k in range(problem.d):
            x, _ = op.nodes(k)
            cores.append(t.factors[k](x[1:-1]).reshape(1, -1, 1))
        cores[0] = cores[0] * t.coef
        blocks.append(cores)
    return _block_tt(blocks)


def full_solution_cores(problem, op):
    """u* at every GLL node (the full grid, n per dimension): Dirichlet data
    g = u* on the boundary, extended by u* itself inside."""
    blocks = []
    for t in problem.terms:
        cores = []
        for k in range(problem.d):
            x, _ = op.nodes(k)
            cores.append(t.factors[k](x).reshape(1, -1, 1))
        cores[0] = cores[0] * t.coef
        blocks.append(cores)
    return _block_tt(blocks)


def build_operator(problem, stream=None):
    from . import t2s2_build_operator
    return t2s2_build_operator(problem.d, problem.n, problem.beta, problem.eps,
                               problem.plain_sc, stream)


def spacetime_dims(st):
    """The per-dimension node data of a space-time workload, time first, from
    the library's host-side t2s2_dim_matrices (no device involved)."""
    from . import DIM_SPACE, DIM_SPACE_PLAIN, DIM_TIME, t2s2_dim_matrices
    sp = st.space
    dims = [t2s2_dim_matrices(st.n_t, 0.0, 2.0 / st.T, DIM_TIME)]
    kind = DIM_SPACE_PLAIN if sp.plain_sc else DIM_SPACE
    dims += [t2s2_dim_matrices(sp.n[k], sp.eps, float(sp.beta[k]), kind) for k in range(sp.d)]
    return dims


def spacetime_source_cores(st, dims):
    """b = (2/T) du*/ds - eps Laplace u* + beta . grad u* on the space-time
    collocation grid (Gauss times, superconsistent points), before the
    initial condition is lifted: per separable term, the spatial source times
    phi_t at the collocation times plus (2/T) phi_t' times the spatial values.
    ``dims`` is ``spacetime_dims(st)``."""
    sp = st.space
    scale = 2.0 / st.T
    g = dims[0]["eta"]
    blocks = []
    for t, ft in zip(sp.terms, st.time_factors):
        one = dataclasses.replace(sp, terms=[t])
        spatial = _sampled_source(one, [dims[k + 1]["eta"] for k in range(sp.d)])
        mass = [t.factors[k](dims[k + 1]["eta"]).reshape(1, -1, 1) for k in range(sp.d)]
        mass[0] = mass[0] * t.coef
        blocks.append([ft(g).reshape(1, -1, 1)] + spatial)
        blocks.append([(scale * ft(g, 1)).reshape(1, -1, 1)] + mass)
    return _block_tt(blocks)


def spacetime_initial_cores(st, dims):
    """u0 = u*(x, s = -1) at the interior spatial GLL nodes (d cores)."""
    sp = st.space
    blocks = []
    for t, ft in zip(sp.terms, st.time_factors):
        cores = [t.factors[k](dims[k + 1]["x"][1:-1]).reshape(1, -1, 1) for k in range(sp.d)]
        cores[0] = cores[0] * (t.coef * float(ft(np.array([-1.0]))[0]))
        blocks.append(cores)
    return _block_tt(blocks)


def _sampled_source(problem, etas):
    """source_cores of ``problem`` at the given collocation points per dimension."""
    class _Nodes:
        def nodes(self, k):
            return None, etas[k]
    return source_cores(problem, _Nodes())
