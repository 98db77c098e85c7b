"""Pins of the stability-map oracle (Results, "Superconsistent
Stabilization"; the stability-domain figure)."""
import numpy as np
import pytest

import workloads as W
from oracle import stability as ST
from oracle import tt as T


def test_sign_change_counter_on_known_sequences():
    assert ST.sign_changes([0, 1, 2, 3]) == 0
    assert ST.sign_changes([0, 1, 2, 1, 0]) == 1
    assert ST.sign_changes([0, 1, 1, 1, 0]) == 1          # flat steps are skipped
    assert ST.sign_changes([0, 2, 1, 2, 1, 2, 0]) == 5
    # brute force against products of neighbouring differences
    for k in range(1, 6):
        v = [0.0] + [1.0 + (i % 2) for i in range(2 * k)] + [0.0]
        dv = np.diff(v)
        brute = sum(1 for a, b in zip(dv[:-1], dv[1:]) if a * b < 0)
        assert ST.sign_changes(v) == brute


def test_tv_excess_on_known_sequences():
    assert ST.tv_excess([0, 1, 2, 1, 0]) == 0.0
    assert ST.tv_excess([0, 0, 0]) == 0.0
    # one overshoot of size 1 on a peak of 2: TV 6 over 4, excess 0.5
    assert abs(ST.tv_excess([0, 2, 1, 2, 0]) - 0.5) < 1e-15


def test_tt_line_equals_the_dense_line():
    cores = W.random_tt(3, 7, [1, 2, 3, 1], seed=1)
    full = T.full(cores)
    assert np.allclose(ST.tt_line(cores), ST.mid_axis_line(full))
    assert np.allclose(ST._fibre(cores), ST.mid_axis_line(full))


@pytest.mark.parametrize("plain", [True, False])
def test_diffusion_dominated_pixels_are_regular(plain):
    for n in (9, 17, 25):
        c = ST.classify(ST.dense_pixel(2, n, 0.1, plain))
        assert not c["oscillatory"] and not c["macroscopic"], (n, c)


def test_plain_sc_oscillates_at_small_ratios():
    for n in (9, 17, 25):
        for ratio in (1e-3, 1e-5):
            c = ST.classify(ST.dense_pixel(2, n, ratio, True))
            assert c["oscillatory"] and c["macroscopic"], (n, ratio, c)


def test_plain_sc_stable_region_grows_with_the_degree():
    # at a fixed ratio, enough degrees make diffusion (~N^4) dominate
    # transport (~N^2): low degrees oscillate, high ones do not
    ratio = 1e-2
    assert ST.classify(ST.dense_pixel(2, 9, ratio, True))["oscillatory"]
    assert ST.classify(ST.dense_pixel(2, 17, ratio, True))["oscillatory"]
    for n in (25, 33):
        assert not ST.classify(ST.dense_pixel(2, n, ratio, True))["oscillatory"]


def test_superconsistent_has_no_macroscopic_oscillation_where_plain_sc_does():
    for n in (9, 17, 25):
        for ratio in (1e-3, 1e-5):
            sc = ST.classify(ST.dense_pixel(2, n, ratio, False))
            pl = ST.classify(ST.dense_pixel(2, n, ratio, True))
            assert pl["macroscopic"] and not sc["macroscopic"], (n, ratio, sc, pl)
            assert sc["tv_excess"] < 0.1 * pl["tv_excess"]
