"""Host-side input preparation for the library (no method arithmetic on the device path).

Samples a workload's analytic factors at the nodes the library reports
(t2s2_op_nodes) and lays them out as TT cores:

* ``source_cores``: b = -eps Laplace u* + beta . grad u* on the collocation
  grid, built exactly from separable terms (the paper derives sources from
  analytic solutions, Results "Global Accuracy"); one rank-2 block per term.
* ``solution_cores``: u* (or an initial condition) on the interior GLL grid,
  one rank-1 block per term.
"""
from __future__ import annotations

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


def build_operator(problem, stream=None):
    from . import t2s2_build_operator
    return t2s2_build_operator(problem.d, problem.n, problem.beta, problem.eps,
                               problem.plain_sc, stream)
