"""Host-side input generation: seeded configs and the warm-start feature map."""
import numpy as np

import workloads as W


def test_warm_features_have_a_fixed_width():
    for d in (3, 4, 6, 7):
        f = W.warm_features(W.config4(123, d=d, n=16))
        assert f.shape == (W.WARM_IN_DIM,) and f.dtype == np.float32
        assert np.all(np.isfinite(f)) and np.max(np.abs(f)) <= 2.0


def test_warm_features_follow_the_parameters():
    p = W.config4(7)
    f = W.warm_features(p)
    ratio = p.eps / (W.EDGE_LENGTH * np.linalg.norm(p.beta))
    assert abs(f[0] - (np.log10(ratio) + 3.0)) < 1e-6
    assert np.allclose(f[1:7], p.beta, atol=1e-7)
    assert np.allclose(f[7:11], (p.params[:4] - 0.75) * 4.0, atol=1e-6)


def test_configs_are_seeded():
    a, b = W.config4(11), W.config4(11)
    assert np.array_equal(a.beta, b.beta) and a.eps == b.eps and np.array_equal(a.params, b.params)
    assert not np.array_equal(W.config4(12).beta, a.beta)


FACTORS = [W.Factor("sine", m=3), W.Factor("wsine", m=2), W.Factor("gauss", mu=0.2, s=0.3),
           W.Factor("wgauss", mu=-0.1, s=0.25), W.Factor("exp", m=1.3),
           W.Factor("poly", c=(0.5, -1.0, 2.0, 0.25))]


def test_factor_derivatives_match_central_differences():
    # every analytic factor's first and second derivatives against fourth-order
    # central differences of its values (step 1e-3: truncation ~1e-12 x f^(5))
    x = np.linspace(-0.9, 0.9, 13)
    h = 1e-3
    for f in FACTORS:
        v = [f(x + k * h) for k in (-2, -1, 0, 1, 2)]
        d1 = (v[0] - 8 * v[1] + 8 * v[3] - v[4]) / (12 * h)
        d2 = (-v[0] + 16 * v[1] - 30 * v[2] + 16 * v[3] - v[4]) / (12 * h * h)
        scale = max(1.0, np.max(np.abs(f(x, 2))))
        assert np.max(np.abs(f(x, 1) - d1)) <= 1e-6 * scale, f
        assert np.max(np.abs(f(x, 2) - d2)) <= 1e-4 * scale, f


def test_boundary_vanishing_factors_vanish():
    for f in (W.Factor("sine", m=1), W.Factor("sine", m=4), W.Factor("wsine", m=3),
              W.Factor("wgauss", mu=0.3, s=0.2)):
        assert np.max(np.abs(f(np.array([-1.0, 1.0])))) < 1e-14


def test_poly_and_exp_closed_forms():
    x = np.array([-1.0, 0.0, 0.5, 1.0])
    p = W.Factor("poly", c=(1.0, 0.0, -1.0))           # 1 - x^2
    assert np.allclose(p(x), 1 - x * x) and np.allclose(p(x, 1), -2 * x) and np.allclose(p(x, 2), -2.0)
    assert np.allclose(W.Factor("poly", c=(3.0,))(x, 1), 0.0)
    e = W.Factor("exp", m=-0.5)
    assert np.allclose(e(x), np.exp(-0.5 * x)) and np.allclose(e(x, 2), 0.25 * np.exp(-0.5 * x))
