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
