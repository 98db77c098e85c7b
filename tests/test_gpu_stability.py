"""GPU parity of the stability map (row N2; Results, "Superconsistent
Stabilization") against the oracle's dense pixels, and of t2s2_tt_fibre
against the oracle's full tensors."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import stability as OS
from oracle import tt as OT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2506_04732_gb300 as pkg
    torch.cuda.set_device(0)
    return pkg


def test_fibre_matches_full_tensor(T):
    from paper_2506_04732_gb300 import problem as P
    op = P.build_operator(W.config1(d=4, n=9))
    cores = W.random_tt(4, 7, [1, 3, 5, 2, 1], seed=3)
    x = T.TT.from_cores(cores)
    full = OT.full(cores)
    rng = np.random.default_rng(4)
    for mode in range(4):
        idx = [int(v) for v in rng.integers(0, 7, 4)]
        got = T.t2s2_tt_fibre(op, x, mode, idx)
        sl = tuple(slice(None) if k == mode else idx[k] for k in range(4))
        assert np.allclose(got, full[sl], rtol=0, atol=1e-14 * np.abs(full).max())
    with pytest.raises(T.T2S2Error):
        T.t2s2_tt_fibre(op, x, 4, [0] * 4)
    with pytest.raises(T.T2S2Error):
        T.t2s2_tt_fibre(op, x, 0, [0, 7, 0, 0])


def test_batched_map_matches_dense_pixels(T):
    from paper_2506_04732_gb300 import stability as S
    d, degrees, ratios = 3, (8, 16), (1e-1, 1e-3)
    pixels, infos = S.solve_map(T, d, degrees, ratios, tol=1e-10, rmax=48, max_sweeps=40, workers=4)
    for (N, r, plain), px in pixels.items():
        assert px["residual"] <= 1e-9, (N, r, plain, px["residual"])
        want = OS.dense_pixel(d, N + 1, r, plain)
        got = np.asarray(px["line"])
        assert np.max(np.abs(got - want)) <= 1e-6 * np.max(np.abs(want)), (N, r, plain)
        c = OS.classify(want)
        assert px["sign_changes"] == c["sign_changes"], (N, r, plain)
        assert abs(px["tv_excess"] - c["tv_excess"]) <= 1e-5
    # the figure's contrast at the small ratio: Plain-SC oscillates
    # macroscopically, the superconsistent scheme does not
    for N in degrees:
        assert pixels[(N, 1e-3, True)]["tv_excess"] > 0.1
        assert pixels[(N, 1e-3, False)]["tv_excess"] < 0.1
