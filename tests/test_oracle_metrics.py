"""Pins for the level-matching measures that every spacing-unit comparison uses.

On an evenly spaced spectrum the local mean spacing is the spacing itself, so errors in spacing
units are exact fractions; a duplicated level or a value far from every level must be reported.
"""

import numpy as np
import pytest

from oracle import metrics as MT


def test_central_exact_takes_smallest_magnitudes_sorted():
    spec = np.array([3.0, -0.5, 0.2, -2.0, 0.9, -0.1])
    assert np.array_equal(MT.central_exact(spec, 3), np.array([-0.5, -0.1, 0.2]))
    assert np.array_equal(MT.central_exact(spec, 6), np.sort(spec))


def test_local_spacing_on_an_even_grid():
    spec = np.arange(-50, 51) * 0.25
    for idx in (0, 3, 50, 99, 100):                 # edges use the one-sided window
        assert MT.local_spacing(spec, idx) == pytest.approx(0.25)
    uneven = np.concatenate([np.arange(0, 10) * 1.0, 10 + np.arange(1, 11) * 3.0])
    # +-10 levels around index 10 reach from level 0 (0.0) to the last, level 19 (40.0): 19 gaps
    assert MT.local_spacing(uneven, 10) == pytest.approx(40.0 / 19)


def test_match_errors_in_spacing_units():
    spec = np.arange(-50, 51) * 0.5
    comp = spec[45:56] + 0.05 * np.linspace(-1, 1, 11)   # shifts of up to a tenth of a spacing
    mt = MT.match(comp, spec)
    assert mt["n_unmatched"] == 0
    assert np.allclose(mt["spacing_err"], np.abs(0.05 * np.linspace(-1, 1, 11)) / 0.5)
    assert np.array_equal(mt["idx"], np.arange(45, 56))


def test_match_reports_duplicates_and_ghosts():
    spec = np.arange(-20, 21) * 1.0
    dup = np.array([-1.0, 0.02, -0.02, 1.0])          # two values on the level 0
    assert MT.match(dup, spec)["n_unmatched"] == 1
    gap = np.array([-2.0, -1.0, 0.0, 1.0, 2.0, 10.0, 11.0, 12.0])
    ghost = np.array([0.0, 5.5])                       # 3.5 from the nearest level, local spacing 2
    mt = MT.match(ghost, gap)
    assert mt["n_unmatched"] == 1 and mt["spacing_err"][1] == pytest.approx(3.5 / 2.0)
