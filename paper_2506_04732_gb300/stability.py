"""Stability map of Plain-SC against superconsistent collocation, run through
the batched solve (Results, "Superconsistent Stabilization", the
stability-domain figure).

Each pixel (polynomial degree N, ratio eps / |beta L|) is the steady problem
-eps Laplace u + beta . grad u = 1 on [-1, 1]^d with beta = (1, .., 1) and
zero Dirichlet data, solved once with collocation at the GLL points
(Plain-SC) and once at the superconsistent points.  All pixels of both
schemes go to t2s2_solve_batched in one call; each solution is read along the
mid-axis in the first direction (the other coordinates at their centre-most
degree of freedom) by t2s2_tt_fibre.  The line is classified by the sign
changes of its consecutive differences (the regular solution rises, then
falls in the outflow layer: one change) and by its total-variation excess
(total variation over 2 max|u|, minus one), large for macroscopic
oscillation.
"""
from __future__ import annotations

import numpy as np

EDGE_LENGTH = 2.0


def line_sign_changes(v) -> int:
    """How often the sign of v[i+1] - v[i] flips (zero steps ignored)."""
    steps = [b - a for a, b in zip(v[:-1], v[1:]) if b != a]
    return sum(1 for s0, s1 in zip(steps[:-1], steps[1:]) if (s0 > 0) != (s1 > 0))


def line_tv_excess(v) -> float:
    """Total variation over twice the largest magnitude, minus one."""
    top = max(abs(float(t)) for t in v)
    if top == 0.0:
        return 0.0
    return sum(abs(float(b) - float(a)) for a, b in zip(v[:-1], v[1:])) / (2.0 * top) - 1.0


def solve_map(T, d, degrees, ratios, tol=1e-8, rmax=30, max_sweeps=30, workers=8):
    """Solve every (degree, ratio) pixel in both schemes with one batched call.

    Returns (pixels, infos): pixels[(N, ratio, plain)] = {"line", "sign_changes",
    "tv_excess", "residual", "sweeps"}."""
    keys, ops, bs, xs = [], [], [], []
    beta = [1.0] * d
    eps_of = {r: r * np.sqrt(d) * EDGE_LENGTH for r in ratios}
    for N in degrees:
        n = N + 1
        for r in ratios:
            for plain in (True, False):
                op = T.t2s2_build_operator(d, [n] * d, beta, eps_of[r], plain)
                m = n - 2
                keys.append((N, r, plain))
                ops.append(op)
                bs.append(T.TT.from_cores([np.ones((1, m, 1))] * d))
                xs.append(T.TT.from_cores([np.ones((1, m, 1))] * d, rcap=rmax + T.RANK_KICK))
    infos = T.t2s2_solve_batched(ops, bs, xs, tol, rmax, max_sweeps, workers=workers, allow_noconv=True)
    pixels = {}
    for key, op, x, info in zip(keys, ops, xs, infos):
        idx = [0] + [m // 2 for m in x.m[1:]]
        v = [0.0] + list(T.t2s2_tt_fibre(op, x, 0, idx)) + [0.0]
        pixels[key] = {"line": v, "sign_changes": line_sign_changes(v), "tv_excess": line_tv_excess(v),
                       "residual": info.residual, "sweeps": info.sweeps}
    return pixels, infos
