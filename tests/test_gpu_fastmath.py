"""The FP64 reciprocal and reciprocal square root of the small factorisations
(binary32 seed, two binary64 Newton steps; IEEE operations outside the binary32
normal range), checked directly against correctly rounded host results.

Bound.  The binary32 seeds carry a relative error e0 of at most a few 2^-23;
each Newton step maps e to about 1.5 e^2 (rsqrt) or e^2 (rcp), so after two
steps the iteration error is below 1e-25 and only the rounding of the last
step's few binary64 operations remains: a few units in the last place.  The
test allows 4 ulp (relative 4 * 2^-53 ~ 4.4e-16) against 1/sqrt(x) and 1/x
formed in binary64 on the host, which carry at most one and a half ulp of
their own.  Inputs cover many decades, both signs for the reciprocal, the
edges of the range where the seed is used (1e-36 and 1e36, just inside and
just outside), zero, infinity and subnormals.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ULP = 2.0 ** -53


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2506_04732_gb300 as pkg
    torch.cuda.set_device(0)
    return pkg


def _inputs():
    rng = np.random.default_rng(2506)
    wide = 10.0 ** rng.uniform(-300, 300, 20000)
    near = 10.0 ** rng.uniform(-40, 40, 20000)
    unit = rng.uniform(0.5, 2.0, 20000)
    edges = np.array([1e-36, 1e36, np.nextafter(1e-36, 1), np.nextafter(1e-36, 0), np.nextafter(1e36, 0),
                      np.nextafter(1e36, np.inf), 1.0000001e-36, 0.9999999e-36, 0.9999999e36, 1.0000001e36,
                      1.0, 2.0, 0.25, 3.0, 1e-300, 1e300, np.finfo(float).max, np.finfo(float).tiny,
                      5e-324, 1e-310])
    return np.concatenate([wide, near, unit, edges])


def test_rsqrt_within_4_ulp_of_correctly_rounded(T):
    x = _inputs()
    rs, _ = T.t2s2_fastmath(torch.tensor(x))
    got = rs.cpu().numpy()
    want = 1.0 / np.sqrt(x)
    rel = np.abs(got - want) / np.abs(want)
    assert np.all(np.isfinite(got))
    assert rel.max() <= 4 * ULP, (x[rel.argmax()], rel.max() / ULP)


def test_rcp_within_4_ulp_of_correctly_rounded_both_signs(T):
    x = _inputs()
    x = np.concatenate([x, -x])
    x = x[np.abs(x) < 1e308]          # 1 / x is representable (not subnormal) below this
    x = x[np.abs(x) > 1e-307]
    _, rc = T.t2s2_fastmath(torch.tensor(x))
    got = rc.cpu().numpy()
    want = 1.0 / x
    rel = np.abs(got - want) / np.abs(want)
    assert rel.max() <= 4 * ULP, (x[rel.argmax()], rel.max() / ULP)


def test_special_values_follow_ieee(T):
    x = np.array([0.0, -0.0, np.inf, -1.0, np.nan])
    rs, rc = T.t2s2_fastmath(torch.tensor(x))
    rs, rc = rs.cpu().numpy(), rc.cpu().numpy()
    assert rs[0] == np.inf and rs[2] == 0.0 and np.isnan(rs[3]) and np.isnan(rs[4])
    assert rc[0] == np.inf and rc[1] == -np.inf and rc[2] == 0.0 and rc[3] == -1.0 and np.isnan(rc[4])
