"""Pins of the oracle's error norms: the max norm and the "L2" norm (root mean square over all
nodes) of the tables of Sec. 5, checked against values worked out by hand and against numpy's
own max and mean; a NaN in the difference must make the max NaN."""
import math

import numpy as np
import pytest


def test_norms_of_a_hand_worked_vector(oracle_mod):
    # |3 - 0|, |-4 - 0|: max 4, rms sqrt((9 + 16) / 2)
    mx, rms = oracle_mod.norms(np.array([3.0, -4.0]))
    assert mx == 4.0
    assert rms == math.sqrt(12.5)
    # a - b with b given: differences (1, -2, 2) -> max 2, rms sqrt(9 / 3) = sqrt(3)
    mx, rms = oracle_mod.norms(np.array([2.0, 0.0, 5.0]), np.array([1.0, 2.0, 3.0]))
    assert mx == 2.0
    assert rms == pytest.approx(math.sqrt(3.0), rel=1e-15)


def test_norms_of_a_constant_vector(oracle_mod):
    # a constant c on N nodes: both norms are |c|, whatever N is
    for n in (1, 7, 1000):
        mx, rms = oracle_mod.norms(np.full(n, -0.375))
        assert mx == 0.375
        assert rms == pytest.approx(0.375, rel=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_norms_match_numpy(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 5000))
    a = rng.standard_normal(n) * 10.0 ** rng.integers(-8, 3)
    b = rng.standard_normal(n)
    d = a - b
    mx, rms = oracle_mod.norms(a, b)
    assert mx == np.max(np.abs(d))
    assert rms == pytest.approx(math.sqrt(np.mean(d * d)), rel=1e-13)
    mx1, rms1 = oracle_mod.norms(a)
    assert mx1 == np.max(np.abs(a))
    assert rms1 == pytest.approx(math.sqrt(np.mean(a * a)), rel=1e-13)


@pytest.mark.parametrize("where", [0, 17, 99])
def test_a_nan_makes_both_norms_nan(oracle_mod, where):
    a = np.linspace(-1.0, 1.0, 100)
    a[where] = np.nan
    mx, rms = oracle_mod.norms(a)
    assert math.isnan(mx) and math.isnan(rms)
    # the NaN in b counts as well, and a large finite value after it does not hide it
    a = np.zeros(100)
    a[-1] = 1e300
    b = np.zeros(100)
    b[where] = np.nan
    mx, rms = oracle_mod.norms(a, b)
    assert math.isnan(mx) and math.isnan(rms)


def test_an_infinite_difference_gives_an_infinite_max(oracle_mod):
    a = np.zeros(10)
    a[3] = -np.inf
    mx, rms = oracle_mod.norms(a)
    assert mx == np.inf and rms == np.inf
