"""Seeded synthetic workloads shaped like the paper's experiments.

This module is shared by the FP64 oracle (``oracle/``) and the GPU library's
tests and benchmark.  It holds problem *parameters* and the analytic 1D factor
functions of manufactured solutions, nothing else: no quadrature nodes, no
collocation matrices, no tensor-train arithmetic.  Each side builds its own
discretisation from these parameters.

Problem statement (Overview, eq. pblm:time:A-C): on the hypercube
Omega = [-1, 1]^d,

    du/dt - eps * Laplace(u) + beta . grad(u) = b,   u = 0 on the boundary.

The steady workloads drop du/dt.  Manufactured solutions follow the Results
section ("Global Accuracy"): the source b is derived analytically from a chosen
u*, here a short sum of separable terms, so b is an exact low-rank TT.

The ratio eps / |beta L| uses L = 2, the edge length of [-1, 1]^d.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = ["Factor", "Term", "Problem", "SpaceTimeProblem", "config0", "config1", "config2",
           "config3", "config4", "config_spacetime", "config_dirichlet", "config_varcoef", "VarCoefProblem", "random_tt", "sine_problem", "random_unit_vector",
           "EDGE_LENGTH"]

EDGE_LENGTH = 2.0


@dataclass(frozen=True)
class Factor:
    """One analytic 1D factor phi(x) of a separable term.

    kind == "sine":   phi(x) = sin(m * pi * (x + 1) / 2)          (vanishes at +-1
                      for integer m)
    kind == "wgauss": phi(x) = (1 - x^2) * exp(-(x - mu)^2 / (2 s^2))
    kind == "gauss":  phi(x) = exp(-(x - mu)^2 / (2 s^2))
    kind == "wsine":  phi(x) = (1 - x^2) * sin(m * pi * x)
    kind == "exp":    phi(x) = exp(m * x)
    kind == "poly":   phi(x) = sum_i c[i] x^i
    """
    kind: str
    m: float = 1.0
    mu: float = 0.0
    s: float = 1.0
    c: tuple = ()

    def __call__(self, x, deriv: int = 0):
        x = np.asarray(x, dtype=np.float64)
        if self.kind == "sine":
            k = self.m * math.pi / 2.0
            t = k * (x + 1.0)
            if deriv == 0:
                return np.sin(t)
            if deriv == 1:
                return k * np.cos(t)
            if deriv == 2:
                return -k * k * np.sin(t)
        elif self.kind == "wsine":
            k = self.m * math.pi
            sn, cs = np.sin(k * x), np.cos(k * x)
            w, w1 = 1.0 - x * x, -2.0 * x
            if deriv == 0:
                return w * sn
            if deriv == 1:
                return w1 * sn + w * k * cs
            if deriv == 2:
                return -2.0 * sn + 2.0 * w1 * k * cs - w * k * k * sn
        elif self.kind in ("gauss", "wgauss"):
            z = (x - self.mu) / self.s
            g = np.exp(-0.5 * z * z)
            g1 = -z / self.s * g                       # g'
            g2 = (z * z - 1.0) / (self.s * self.s) * g  # g''
            if self.kind == "gauss":
                return (g, g1, g2)[deriv]
            w, w1, w2 = 1.0 - x * x, -2.0 * x, -2.0 * np.ones_like(x)
            if deriv == 0:
                return w * g
            if deriv == 1:
                return w1 * g + w * g1
            if deriv == 2:
                return w2 * g + 2.0 * w1 * g1 + w * g2
        elif self.kind == "exp":
            if deriv in (0, 1, 2):
                return self.m ** deriv * np.exp(self.m * x)
        elif self.kind == "poly":
            if deriv in (0, 1, 2):
                c = np.polynomial.polynomial.polyder(np.asarray(self.c, dtype=np.float64), deriv)
                return np.polynomial.polynomial.polyval(x, c) + 0.0 * x
        raise ValueError(f"bad factor {self.kind} / deriv {deriv}")


@dataclass(frozen=True)
class Term:
    """coef * prod_k factors[k](x_k)."""
    coef: float
    factors: tuple


@dataclass
class Problem:
    """A steady or time-dependent workload on [-1,1]^d with zero Dirichlet data.

    ``n`` is the number of Gauss-Lobatto-Legendre nodes per dimension
    (polynomial degree n-1).  ``terms`` is the manufactured solution u* for
    steady problems, or the initial condition for time-dependent ones.
    """
    name: str
    d: int
    n: tuple
    beta: np.ndarray
    eps: float
    terms: list
    tol: float
    rmax: int
    max_sweeps: int = 50
    plain_sc: bool = False
    dt: float = 0.0
    steps: int = 0
    seed: int = 0
    params: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def ratio(self) -> float:
        """eps / (|beta| L)."""
        return self.eps / (float(np.linalg.norm(self.beta)) * EDGE_LENGTH)


def random_unit_vector(d: int, rng: np.random.Generator) -> np.ndarray:
    v = rng.standard_normal(d)
    return v / np.linalg.norm(v)


def config0() -> Problem:
    """d=3, n=16, beta=(1,1,1)/sqrt(3), eps=1e-2, u* = prod sin(pi (x+1)/2)."""
    d, n = 3, 16
    f = Factor("sine", m=1)
    return Problem("steady d=3 n=16 eps=1e-2", d, (n,) * d,
                   np.ones(d) / math.sqrt(d), 1e-2,
                   [Term(1.0, (f,) * d)], tol=1e-12, rmax=16, max_sweeps=40)


def config1(seed_beta: int = 1, seed_terms: int = 2, d: int = 6, n: int = 32,
            ratio: float = 1e-3, rmax: int = 20, tol: float = 1e-8) -> Problem:
    """d=6, n=32, eps/|beta L| = 1e-3, rank-4 u*: 2 sine + 2 windowed Gaussian terms."""
    beta = random_unit_vector(d, np.random.default_rng(seed_beta))
    eps = ratio * EDGE_LENGTH
    rng = np.random.default_rng(seed_terms)
    terms = []
    for t in range(4):
        c = float(rng.uniform(0.5, 1.0))
        if t < 2:
            fs = tuple(Factor("sine", m=int(rng.integers(1, 5))) for _ in range(d))
        else:
            fs = tuple(Factor("wgauss", mu=float(rng.uniform(-0.5, 0.5)), s=0.3)
                       for _ in range(d))
        terms.append(Term(c, fs))
    return Problem(f"steady d={d} n={n} ratio={ratio:g}", d, (n,) * d, beta, eps,
                   terms, tol=tol, rmax=rmax, max_sweeps=50, seed=seed_terms)


# Full width at half maximum of a Gaussian, in units of its standard deviation.
_FWHM_PER_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))


def config2(seed_beta: int = 3, seed_center: int = 4, d: int = 7, n: int = 64,
            ratio: float = 1e-4, dt: float = 1e-3, steps: int = 100,
            rmax: int = 40, tol: float = 1e-8, width: float = 0.2) -> Problem:
    """Crank-Nicolson workload: separable Gaussian pulse of FWHM ``width``."""
    beta = random_unit_vector(d, np.random.default_rng(seed_beta))
    rng = np.random.default_rng(seed_center)
    s = width / _FWHM_PER_SIGMA
    fs = tuple(Factor("gauss", mu=float(rng.uniform(-0.5, 0.5)), s=s) for _ in range(d))
    return Problem(f"CN d={d} n={n} ratio={ratio:g}", d, (n,) * d, beta,
                   ratio * EDGE_LENGTH, [Term(1.0, fs)], tol=tol, rmax=rmax,
                   max_sweeps=20, dt=dt, steps=steps, seed=seed_center)


def config3(i: int, d: int = 5) -> Problem:
    """Instance i of the batched workload (seed 1000+i)."""
    rng = np.random.default_rng(1000 + i)
    n = int(rng.choice([16, 24, 32, 48]))
    ratio = float(10.0 ** rng.uniform(-4.0, -1.0))
    beta = random_unit_vector(d, rng)
    terms = [Term(1.0, tuple(Factor("sine", m=int(rng.integers(1, 5))) for _ in range(d)))
             for _ in range(2)]
    return Problem(f"batched#{i} d={d} n={n}", d, (n,) * d, beta, ratio * EDGE_LENGTH,
                   terms, tol=1e-8, rmax=16, max_sweeps=50, seed=1000 + i)


def config4(seed: int, d: int = 6, n: int = 32) -> Problem:
    """Warm-start workload: rank-4 u* with 8 scalar parameters.

    Parameters p = (a_1..a_4, w_1, w_2, mu_3, mu_4): amplitudes a_t in [0.5, 1],
    sine frequencies w_t in [1, 3] entering through (1 - x^2) sin(w pi x), and
    Gaussian centres mu_t in [-0.5, 0.5] of windowed Gaussians of width 0.3.
    """
    rng = np.random.default_rng(seed)
    ratio = float(10.0 ** rng.uniform(-4.0, -2.0))
    beta = random_unit_vector(d, rng)
    a = rng.uniform(0.5, 1.0, 4)
    w = rng.uniform(1.0, 3.0, 2)
    mu = rng.uniform(-0.5, 0.5, 2)
    terms = [Term(float(a[0]), tuple(Factor("wsine", m=float(w[0])) for _ in range(d))),
             Term(float(a[1]), tuple(Factor("wsine", m=float(w[1])) for _ in range(d))),
             Term(float(a[2]), tuple(Factor("wgauss", mu=float(mu[0]), s=0.3) for _ in range(d))),
             Term(float(a[3]), tuple(Factor("wgauss", mu=float(mu[1]), s=0.3) for _ in range(d)))]
    p = np.concatenate([a, w, mu])
    return Problem(f"warm#{seed} d={d} n={n}", d, (n,) * d, beta, ratio * EDGE_LENGTH,
                   terms, tol=1e-8, rmax=20, max_sweeps=50, seed=seed, params=p)


WARM_IN_DIM = 15


def warm_features(p: Problem) -> np.ndarray:
    """Input vector of the warm-start network for a config4-style problem.

    15 values, each scaled to about [-1, 1]: log10(eps / (|beta| L)) + 3, the
    components of beta (zero-padded or cut to 6), the 4 amplitudes
    (a - 0.75) * 4, the 2 frequencies w - 2 and the 2 centres 2 mu.  (An input
    width of 11 cannot hold beta, the diffusion ratio and 8 source parameters
    at d = 6; 15 can.)
    """
    beta = np.asarray(p.beta, dtype=np.float64)
    ratio = p.eps / (EDGE_LENGTH * float(np.linalg.norm(beta)))
    b6 = np.zeros(6)
    b6[:min(6, beta.size)] = beta[:6]
    a, w, mu = p.params[:4], p.params[4:6], p.params[6:8]
    f = np.concatenate([[math.log10(ratio) + 3.0], b6, (a - 0.75) * 4.0, w - 2.0, 2.0 * mu])
    assert f.size == WARM_IN_DIM
    return f.astype(np.float32)


@dataclass
class SpaceTimeProblem:
    """A workload of the unified space-time form: the spatial problem (its
    ``terms`` give the spatial factors), one time factor per term, n_t time
    nodes and the length T of the time interval.
    u*(x, s) = sum_t coef_t phi_t(s) prod_k phi_{t,k}(x_k), s in [-1, 1]."""
    space: Problem
    time_factors: tuple
    n_t: int
    T: float


def config_spacetime(seed: int = 6, d: int = 5, n: int = 32, n_t: int = 24, T: float = 1.0,
                     ratio: float = 1e-3, tol: float = 1e-8, rmax: int = 20) -> SpaceTimeProblem:
    """Space-time workload (time as the first collocated dimension): two
    separable sine terms in space, growing and decaying exponentials in time."""
    rng = np.random.default_rng(seed)
    beta = random_unit_vector(d, rng)
    terms = [Term(1.0, tuple(Factor("sine", m=int(rng.integers(1, 4))) for _ in range(d))),
             Term(0.5, tuple(Factor("sine", m=int(rng.integers(1, 4))) for _ in range(d)))]
    sp = Problem(f"space-time d={d}+1 n={n} n_t={n_t} ratio={ratio:g}", d, (n,) * d, beta,
                 ratio * EDGE_LENGTH, terms, tol=tol, rmax=rmax, max_sweeps=30, seed=seed)
    return SpaceTimeProblem(sp, (Factor("exp", m=1.0), Factor("exp", m=-0.7)), n_t, T)


def config_dirichlet(seed: int = 8, d: int = 5, n: int = 24, ratio: float = 1e-2, tol: float = 1e-8,
                     rmax: int = 20) -> Problem:
    """Non-zero Dirichlet data (u = g on the boundary, g = u* there): u* is a
    sum of two separable terms that do not vanish at +-1, exponentials
    exp(a x) with a in [-1, 1] and Gaussians of width 0.6 centred in
    [-0.5, 0.5].  The source b = -eps Laplace u* + beta . grad u* as for the
    other workloads."""
    rng = np.random.default_rng(seed)
    beta = random_unit_vector(d, rng)
    terms = [Term(1.0, tuple(Factor("exp", m=float(rng.uniform(-1.0, 1.0))) for _ in range(d))),
             Term(0.5, tuple(Factor("gauss", mu=float(rng.uniform(-0.5, 0.5)), s=0.6) for _ in range(d)))]
    return Problem(f"dirichlet d={d} n={n} ratio={ratio:g}", d, (n,) * d, beta, ratio * EDGE_LENGTH,
                   terms, tol=tol, rmax=rmax, max_sweeps=30, seed=seed)


@dataclass
class VarCoefProblem:
    """Variable coefficients for a Problem: beta_k(x) = beta_ref[k] (1 + a_k
    sin(pi x)) and rho(x) = rho0 + sum_k c_k (1 + x_k^2); beta_ref[k] (the
    problem's beta) is the speed that picks the superconsistent points."""
    problem: Problem
    amp: np.ndarray
    rho_c: np.ndarray
    rho0: float
    prod: bool = False

    def beta_fn(self, k):
        b, a = float(self.problem.beta[k]), float(self.amp[k])
        return lambda x: b * (1.0 + a * np.sin(np.pi * np.asarray(x, dtype=np.float64)))

    def rho_fn(self, k):
        c = float(self.rho_c[k])
        return lambda x: c * (1.0 + np.asarray(x, dtype=np.float64) ** 2)

    @staticmethod
    def prod_fn(k):
        """One factor of the paper's product reaction, the same in every
        dimension: 1/2 - (x + 11/10)(x - 1/2)(x + 1/2)(x - 11/10)."""
        def f(x):
            x = np.asarray(x, dtype=np.float64)
            return 0.5 - (x + 1.1) * (x - 0.5) * (x + 0.5) * (x - 1.1)
        return f


def config_varcoef(seed: int = 9, d: int = 6, n: int = 32, ratio: float = 1e-3, tol: float = 1e-8,
                   rmax: int = 20, prod: bool = False) -> VarCoefProblem:
    """Variable convection beta_k(x_k) (amplitudes a_k in [0.2, 0.5] around a
    seeded unit vector) and reaction rho0 + sum_k c_k (1 + x_k^2) (rho0 = 0.5,
    c_k in [0, 0.3]), plus with `prod` the paper's product reaction
    prod_k (1/2 - (x_k + 11/10)(x_k - 1/2)(x_k + 1/2)(x_k - 11/10)); u* the
    rank-4 recipe of config1 with the same seed."""
    base = config1(seed_beta=seed, seed_terms=seed + 1, d=d, n=n, ratio=ratio, rmax=rmax, tol=tol)
    base.name = f"varcoef{'+prod' if prod else ''} d={d} n={n} ratio={ratio:g}"
    rng = np.random.default_rng(seed + 2)
    return VarCoefProblem(base, rng.uniform(0.2, 0.5, d), rng.uniform(0.0, 0.3, d), 0.5, prod)


def sine_problem(d: int, n: int, ratio: float, seed: int = 5, tol: float = 1e-8,
                 rmax: int = 12) -> Problem:
    """Small well-resolved steady problem: u* = prod sin(pi(x+1)/2) + 0.5 prod sin(pi(x+1))."""
    beta = random_unit_vector(d, np.random.default_rng(seed))
    terms = [Term(1.0, (Factor("sine", m=1),) * d), Term(0.5, (Factor("sine", m=2),) * d)]
    return Problem(f"sines d={d} n={n} ratio={ratio:g}", d, (n,) * d, beta, ratio * EDGE_LENGTH,
                   terms, tol=tol, rmax=rmax, max_sweeps=30, seed=seed)


def random_tt(d: int, n, ranks, seed: int, dtype=np.float64):
    """Random TT cores G_k of shape (r_{k-1}, n_k, r_k), entries N(0,1)/sqrt(r_{k-1} n_k).

    ``ranks`` has d+1 entries with ranks[0] == ranks[d] == 1.
    """
    if np.isscalar(n):
        n = (int(n),) * d
    assert len(ranks) == d + 1 and ranks[0] == 1 and ranks[-1] == 1
    rng = np.random.default_rng(seed)
    cores = []
    for k in range(d):
        a, m, b = ranks[k], n[k], ranks[k + 1]
        cores.append((rng.standard_normal((a, m, b)) / math.sqrt(a * m)).astype(dtype))
    return cores
