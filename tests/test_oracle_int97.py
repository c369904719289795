"""Pins of the reversible integer CDF 9/7 (dyadic Table I steps: a = -3/2,
b = -1/16, g = 205/256, d = 15/32; updates rounded with floor(c s + 1/2);
diagonal scalings dropped)."""
import numpy as np
import pytest


def test_hand_computed_level_with_floor_rounding(oracle):
    """K = 4, x side, worked by hand: the g step sees -205/256 + 1/2 = -77/256,
    which floors to -1 (truncation would give 0)."""
    a, b = oracle.int97_level(0, [-3, 5, 2, -7])
    assert a.tolist() == [-3, 2] and b.tolist() == [6, -6]


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("K", [2, 4, 6, 64, 1000])
def test_reversible(oracle, side, K):
    g = np.random.default_rng(K + side)
    v = g.integers(-32768, 32768, size=K)
    a, b = oracle.int97_level(side, v)
    np.testing.assert_array_equal(oracle.int97_level_inv(side, a, b), v)


@pytest.mark.parametrize("side", [0, 1])
def test_tracks_the_float_steps(oracle, side):
    """The rounded steps stay within a few units of the same steps in exact
    arithmetic (dyadic constants, no scaling)."""
    g = np.random.default_rng(5 + side)
    K = 256
    v = g.integers(-20000, 20000, size=K).astype(np.float64)
    e, o = v[0::2].copy(), v[1::2].copy()
    c = np.array([-1.5, -1.0 / 16, 205.0 / 256, 15.0 / 32])
    for s in range(4):
        odd = (s % 2 == 0) if side == 0 else (s % 2 == 1)
        k = c[s] if side == 0 else -c[s]
        if odd:
            o = o + k * (e + np.roll(e, -1))
        else:
            e = e + k * (o + np.roll(o, 1))
    a, b = oracle.int97_level(side, v.astype(np.int64))
    assert np.abs(a - e).max() <= 8 and np.abs(b - o).max() <= 8
