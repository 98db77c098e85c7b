"""Stability map of Plain-SC against superconsistent collocation (oracle;
test infrastructure).

Results, "Superconsistent Stabilization" and the stability-domain figure: the
steady problem -eps Laplace u + beta . grad u = b on [-1, 1]^d with beta a
vector of ones, a constant source (the paper's "identity function" read as
b = 1) and zero Dirichlet data is solved for a grid of (polynomial degree,
eps / |beta L|) pixels, once with collocation at the GLL points (Plain-SC) and
once at the superconsistent points.  A pixel is oscillatory when the first
derivative of the numerical solution, along the mid-axis in the first
direction (the other coordinates at their centre-most degree of freedom),
changes sign more often than that of the regular solution, which rises and
then falls once in the outflow boundary layer: one sign change.

Here the derivative's signs are those of the differences of consecutive
nodal values along that line, the boundary zeros included.  Besides that
count, ``tv_excess`` measures the size of the oscillation: the total
variation of the line over the 2 max|u| of a single rise and fall, minus one
(zero for the regular profile).  A pixel is counted as macroscopically
oscillatory (the figure caption's word for the Plain-SC failures) when the
excess is above 0.1; this threshold is a reading.

Pins (tests/test_oracle_stability.py): the counters on sequences whose
counts are known; in two dimensions, diffusion-dominated pixels regular in
both schemes, Plain-SC oscillating at small ratios, its stable region
growing with the degree at a fixed ratio (diffusive terms grow like N^4,
transport ones like N^2), and the superconsistent solution without
macroscopic oscillation where Plain-SC has it.
"""
from __future__ import annotations

import numpy as np

from . import tt as T
from .collocation import op1d
from .solve import dense_solve

EDGE = 2.0


def pixel_ops(d: int, n: int, ratio: float, plain: bool):
    """1D pieces of one pixel: beta = (1, .., 1), eps = ratio |beta| L."""
    eps = ratio * np.sqrt(d) * EDGE
    return [op1d(n, eps, 1.0, plain) for _ in range(d)]


def ones_source(ops):
    """b = 1 on the collocation grid (a rank-1 TT)."""
    return [np.ones((1, o.n - 2, 1)) for o in ops]


def centre_index(m: int) -> int:
    """The centre-most of m interior degrees of freedom (0-based)."""
    return m // 2


def mid_axis_line(u: np.ndarray) -> np.ndarray:
    """Nodal values along the first direction through the centre-most dof of
    the others, with the boundary zeros at both ends (u: interior array)."""
    idx = (slice(None),) + tuple(centre_index(s) for s in u.shape[1:])
    return np.concatenate([[0.0], u[idx], [0.0]])


def sign_changes(v: np.ndarray) -> int:
    """Sign changes of the consecutive differences of v (zero differences skipped)."""
    dv = np.diff(np.asarray(v, dtype=np.float64))
    s = np.sign(dv[dv != 0.0])
    return int(np.count_nonzero(s[1:] != s[:-1]))


def tv_excess(v: np.ndarray) -> float:
    """Total variation of v over 2 max|v|, minus one."""
    v = np.asarray(v, dtype=np.float64)
    peak = np.max(np.abs(v))
    if peak == 0.0:
        return 0.0
    return float(np.sum(np.abs(np.diff(v))) / (2.0 * peak) - 1.0)


def classify(v: np.ndarray, expected: int = 1, macro: float = 0.1):
    c = sign_changes(v)
    e = tv_excess(v)
    return {"sign_changes": c, "oscillatory": c > expected, "tv_excess": e, "macroscopic": e > macro}


def dense_pixel(d: int, n: int, ratio: float, plain: bool):
    """The mid-axis line of one pixel from the dense solve (tiny grids)."""
    ops = pixel_ops(d, n, ratio, plain)
    u = dense_solve(ops, ones_source(ops))
    return mid_axis_line(u)


def tt_line(cores) -> np.ndarray:
    """The mid-axis line of a TT solution (interior cores)."""
    return mid_axis_line(T.full(cores)) if np.prod([c.shape[1] for c in cores]) <= 2_000_000 else _fibre(cores)


def _fibre(cores):
    r = np.ones((1,))
    for c in reversed(cores[1:]):
        r = c[:, centre_index(c.shape[1]), :] @ r
    v = cores[0][0] @ r
    return np.concatenate([[0.0], v, [0.0]])
