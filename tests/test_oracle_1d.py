"""Pins for the oracle's 1D pieces: GLL points, superconsistent points, R/D/D2.

Each test checks the oracle against something other than itself: textbook
closed forms, numpy's independent Legendre-series routines, exact polynomial
calculus, and the properties the paper states in Overview (i)-(ii) and Fig. 1.
"""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly

from oracle.gll import gauss_nodes, gll_nodes, legendre
from oracle.collocation import lagrange_matrices, op1d, sc_nodes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gll_closed_forms():
    with open(os.path.join(GOLDEN, "gll_closed_forms.json")) as f:
        cases = json.load(f)["cases"]
    env = {"sqrt": math.sqrt}
    for c in cases:
        x, w = gll_nodes(c["N"])
        xe = np.array([eval(s, env) for s in c["nodes"]])
        we = np.array([eval(s, env) for s in c["weights"]])
        assert np.allclose(x, xe, atol=1e-15, rtol=0)
        assert np.allclose(w, we, atol=1e-15, rtol=0)


@pytest.mark.parametrize("N", [2, 3, 5, 8, 15, 31, 47, 63])
def test_gll_nodes_against_numpy_series_roots(N):
    x, _ = gll_nodes(N)
    ref = np.sort(npleg.Legendre.basis(N).deriv().roots().real)
    assert np.max(np.abs(x[1:-1] - ref)) < 1e-13
    assert x[0] == -1.0 and x[-1] == 1.0
    assert np.allclose(x, -x[::-1], atol=1e-15)


@pytest.mark.parametrize("N", [2, 4, 9, 15, 31, 63])
def test_gll_quadrature_exactness(N):
    x, w = gll_nodes(N)
    assert abs(w.sum() - 2.0) < 1e-13
    for m in range(0, 2 * N):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.dot(w, x ** m) - exact) < 1e-13
    # degree 2N is not integrated exactly: GLL gives sum w P_N^2 = 2/N, not 2/(2N+1)
    pN, _, _ = legendre(N, x)
    assert abs(np.dot(w, pN * pN) - 2.0 / N) < 1e-13


@pytest.mark.parametrize("N", [2, 7, 16, 40, 63])
def test_gauss_nodes_against_numpy(N):
    g = gauss_nodes(N)
    assert np.max(np.abs(np.sort(g) - npleg.leggauss(N)[0])) < 1e-14


def test_legendre_recurrence_against_numpy():
    xs = np.linspace(-1, 1, 101)
    for N in [0, 1, 2, 5, 17, 63]:
        p, d1, d2 = legendre(N, xs)
        ser = npleg.Legendre.basis(N)
        assert np.allclose(p, ser(xs), atol=1e-13)
        assert np.allclose(d1, ser.deriv(1)(xs), atol=1e-10 * max(1, N * N))
        assert np.allclose(d2, ser.deriv(2)(xs), atol=1e-10 * max(1, N ** 4))


def test_sc_node_closed_form_degree2():
    # N = 2: q = 3 eps x - beta (3x^2 - 1)/2; keep the root away from the outflow end.
    for eps, beta in [(1.0, 1.0), (1e-3, 1.0), (0.3, -2.0), (5.0, 0.7)]:
        eta = sc_nodes(2, eps, beta)
        # roots (eps -+ sqrt(eps^2 + beta^2/3)) / beta; the kept one is away from x = sign(beta)
        exact = (eps - math.sqrt(eps * eps + beta * beta / 3.0)) / beta
        assert eta.shape == (1,)
        assert abs(eta[0] - exact) < 1e-14


@pytest.mark.parametrize("N", [4, 7, 15, 31, 63])
def test_sc_limit_diffusion_dominated(N):
    # eps/|beta| -> infinity: the zeros of P_N' (Overview (ii)).
    x, _ = gll_nodes(N)
    for ratio in [1e6, 1e9]:
        eta = sc_nodes(N, ratio, 1.0)
        assert np.max(np.abs(eta - x[1:-1])) < 10.0 / ratio


@pytest.mark.parametrize("N", [4, 7, 15, 31, 63])
def test_sc_limit_convection_dominated(N):
    # eps/|beta| -> 0: N-1 of the N zeros of P_N; the one at the outflow end drops.
    g = np.sort(npleg.leggauss(N)[0])
    for ratio in [1e-9, 1e-12]:
        assert np.max(np.abs(sc_nodes(N, ratio, 1.0) - g[:-1])) < 1e3 * ratio * N * N
        assert np.max(np.abs(sc_nodes(N, ratio, -1.0) - g[1:])) < 1e3 * ratio * N * N


@pytest.mark.parametrize("N", [3, 8, 20, 47])
def test_sc_depends_on_ratio_only_and_mirror(N):
    for ratio in [1e-4, 1e-2, 0.3, 10.0]:
        a = sc_nodes(N, ratio, 1.0)
        b = sc_nodes(N, 7.5 * ratio, 7.5)
        c = sc_nodes(N, ratio, -1.0)
        assert np.max(np.abs(a - b)) < 1e-13
        assert np.max(np.abs(a + c[::-1])) < 1e-13


@pytest.mark.parametrize("N", [3, 8, 20, 47])
def test_sc_nodes_interlace_gauss_and_gll(N):
    # beta > 0: eta_j lies between the j-th Gauss point and the j-th interior GLL point.
    x, _ = gll_nodes(N)
    g = np.sort(npleg.leggauss(N)[0])
    for ratio in [1e-5, 1e-3, 1e-1, 10.0]:
        eta = sc_nodes(N, ratio, 1.0)
        assert np.all(eta > g[:-1] - 1e-14) and np.all(eta < x[1:-1] + 1e-14)


@pytest.mark.parametrize("N", [3, 7, 20])
def test_sc_nodes_shift_monotonically_as_diffusion_falls(N):
    # Overview (ii), Fig. 1: with n fixed, lowering eps moves the points steadily
    # from the zeros of P_N' towards the zeros of P_N (for beta > 0: every
    # eta_j decreases monotonically with eps, from x_j towards g_j)
    x, _ = gll_nodes(N)
    g = np.sort(npleg.leggauss(N)[0])
    eps = np.logspace(2, -6, 33)
    etas = np.array([sc_nodes(N, e, 1.0) for e in eps])
    assert np.all(np.diff(etas, axis=0) <= 1e-15)                      # decreasing with eps
    assert np.max(np.abs(etas[0] - x[1:-1])) < 1e-2 * np.max(np.diff(x))   # near P_N' zeros
    assert np.max(np.abs(etas[-1] - g[:-1])) < 1e-2 * np.max(np.diff(x))   # near P_N zeros


def _poly_eval(coef, x, deriv=0):
    return nppoly.polyval(x, nppoly.polyder(coef, deriv) if deriv else coef)


@pytest.mark.parametrize("N", [4, 9, 15, 31])
def test_lagrange_matrices_exact_on_degree_N(N):
    rng = np.random.default_rng(N)
    x, _ = gll_nodes(N)
    eta = sc_nodes(N, 1e-2, 1.0)
    R, D, D2 = lagrange_matrices(x, eta)
    for deg in [0, 1, N // 2, N]:
        c = rng.standard_normal(deg + 1)
        u = _poly_eval(c, x)
        scale = np.max(np.abs(u))
        assert np.max(np.abs(R @ u - _poly_eval(c, eta))) < 1e-12 * scale
        assert np.max(np.abs(D @ u - _poly_eval(c, eta, 1))) < 1e-11 * scale * N * N
        assert np.max(np.abs(D2 @ u - _poly_eval(c, eta, 2))) < 1e-10 * scale * N ** 4


@pytest.mark.parametrize("N", [4, 9, 15, 31, 47])
def test_superconsistency_exact_on_degree_N_plus_1(N):
    # The collocated operator sees grid values only; for u of degree N+1 it still
    # returns (beta u' - eps u'')(eta) exactly at the superconsistent points.
    rng = np.random.default_rng(100 + N)
    x, _ = gll_nodes(N)
    for ratio, beta in [(1e-3, 1.0), (0.05, -0.6), (2.0, 0.3)]:
        eps = ratio * abs(beta)
        o = op1d(N + 1, eps, beta)
        Lfull = beta * o.D - eps * o.D2
        # u in the Legendre basis with an O(1) degree-(N+1) component
        c = rng.standard_normal(N + 2)
        c[-1] = 1.0
        u = npleg.legval(x, c)
        Lu = lambda pts: beta * npleg.legval(pts, npleg.legder(c, 1)) - eps * npleg.legval(pts, npleg.legder(c, 2))
        exact = Lu(o.eta)
        scale = np.max(np.abs(exact)) + np.max(np.abs(u)) * (abs(beta) * N * N + eps * N ** 4)
        assert np.max(np.abs(Lfull @ u - exact)) < 1e-13 * scale
        # at the plain GLL points the same degree-(N+1) exactness fails
        p = op1d(N + 1, eps, beta, plain=True)
        err_plain = np.max(np.abs((beta * p.D - eps * p.D2) @ u - Lu(p.eta)))
        assert err_plain > 1e-3 * abs(beta)


def _adv_diff_exact(x, beta, eps):
    # beta u' - eps u'' = 1, u(+-1) = 0   (eq. adv-diff-1d)
    t = beta / eps
    return (x + 1) / beta - 2.0 / beta * (np.exp(t * (x - 1)) - np.exp(-2 * t)) / (1 - np.exp(-2 * t))


def _sign_changes(v):
    s = np.sign(v[np.abs(v) > 1e-12 * np.max(np.abs(v))])
    return int(np.sum(s[1:] != s[:-1]))


@pytest.mark.parametrize("n", [8, 16, 24, 40])
def test_fig1_adv_diff_sc_stable_plain_oscillates(n):
    # Fig. 1 (c)-(d): in the convection-dominated regime the Plain-SC solution
    # is unreliable while the superconsistent one is not.  The exact solution of
    # eq. adv-diff-1d is positive on (-1, 1) with peak 2 - O(eps) and a derivative
    # that changes sign once.
    beta, eps = 1.0, 1e-5
    sols = {}
    for plain in (False, True):
        o = op1d(n, eps, beta, plain)
        u = np.linalg.solve(o.Lt, np.ones(n - 2))
        full = np.concatenate([[0.0], u, [0.0]])
        fine = np.linspace(-1.0, 1.0, 50 * n + 1)
        _, Dx, _ = lagrange_matrices(o.x, fine)
        sols[plain] = (u, _sign_changes(Dx @ full))
    u_sc, ch_sc = sols[False]
    u_pl, ch_pl = sols[True]
    assert np.min(u_sc) > 0.0
    assert abs(np.max(u_sc) - 2.0) < 0.35
    assert np.min(u_pl) < -0.3            # wrong-signed values
    assert ch_pl >= n - 4                 # oscillation at every node
    assert ch_sc < ch_pl
    # away from the outflow layer the SC solution follows the exact one
    o = op1d(n, eps, beta)
    xi = o.x[1:-1]
    mask = xi < 0.5
    assert np.max(np.abs(u_sc[mask] - _adv_diff_exact(xi[mask], beta, eps))) < 0.05


def test_fig1_balanced_regime_sc_and_plain_agree():
    # Fig. 1(a): when convection and diffusion balance, both solutions almost coincide.
    beta, eps, n = 1.0, 0.5, 16
    us = []
    for plain in (False, True):
        o = op1d(n, eps, beta, plain)
        us.append(np.linalg.solve(o.Lt, np.ones(n - 2)))
    o = op1d(n, eps, beta)
    ex = _adv_diff_exact(o.x[1:-1], beta, eps)
    assert np.max(np.abs(us[0] - ex)) < 1e-10
    assert np.max(np.abs(us[1] - ex)) < 1e-10
