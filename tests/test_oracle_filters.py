"""Pins of the oracle's one-level lifting against what the paper prints.

Each lifting factorisation (eq. 17; Sec. III-C Case I and II with Table I) is
checked against the convolution-and-downsample filterbank built from the
printed filter taps (tests/golden/filters.json), against perfect
reconstruction, against the dual-basis pairing that makes eq. 4 hold, and
against the vanishing moments the paper states for each filter.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from tests import golden_taps as G

FILTERS = [(0, "d4"), (1, "legall53"), (2, "cdf97")]
SIDES = [(0, "x"), (1, "y")]


def impulse_taps(O, f, side, K=64, n0=16):
    lo, hi = {}, {}
    for m in range(-10, 11):
        v = np.zeros(K)
        v[(2 * n0 + m) % K] = 1.0
        a, b = O.lift_level(f, side, v)
        if abs(a[n0]) > 1e-15:
            lo[m] = a[n0]
        if abs(b[n0]) > 1e-15:
            hi[m] = b[n0]
    return lo, hi


@pytest.mark.parametrize("f,name", FILTERS)
@pytest.mark.parametrize("side,sname", SIDES)
def test_lifting_impulse_response_equals_printed_taps(oracle, f, name, side, sname):
    lo, hi = impulse_taps(oracle, f, side)
    elo, ehi = G.filter_taps(name, sname)
    assert set(lo) == set(elo), (lo, elo)
    assert set(hi) == set(ehi), (hi, ehi)
    for m in elo:
        assert lo[m] == pytest.approx(elo[m], abs=1e-14)
    for m in ehi:
        assert hi[m] == pytest.approx(ehi[m], abs=1e-14)


@pytest.mark.parametrize("f,name", FILTERS)
@pytest.mark.parametrize("side,sname", SIDES)
@pytest.mark.parametrize("K", [8, 14, 64, 250])
def test_lifting_equals_mallat_on_random_input(oracle, f, name, side, sname, K):
    g = np.random.default_rng(K + 10 * f + side)
    v = g.standard_normal(K)
    a, b = oracle.lift_level(f, side, v)
    lo, hi = G.filter_taps(name, sname)
    am, bm = oracle.mallat_level(v, lo, hi)
    np.testing.assert_allclose(a, am, rtol=0, atol=1e-13)
    np.testing.assert_allclose(b, bm, rtol=0, atol=1e-13)


def test_eq7_rule_reproduces_printed_legall53_highpasses():
    g = G.load()["legall53"]
    h = G.taps(dict(g["y_lo"], scale="1"))       # h(z), unscaled
    ht = G.taps(g["x_lo"])                       # h~(z^-1)
    assert G.modulated_highpass(h) == pytest.approx(G.taps(g["x_hi"]))
    assert G.modulated_highpass(ht, 2.0) == pytest.approx(G.taps(g["y_hi"]))


def test_cdf97_table1_from_t_formulas(oracle):
    """Sec. III-C Case II: a, b, g, d, x as functions of t; t = 5/4 gives Table I."""
    t = Fraction(5, 4)
    a = (-2 * t + 1) / (4 * (t - 1))
    b = -(t - 1) ** 2
    gg = 1 / (4 * t * (t - 1))
    d = t ** 3 - Fraction(7, 4) * t ** 2 + t
    tab = G.load()["table1"]
    assert (a, b, gg, d) == tuple(Fraction(tab[k]) for k in "abgd")
    c = oracle.cdf97_constants()
    assert tuple(c[:4]) == (float(a), float(b), float(gg), float(d))
    assert c[4] == pytest.approx(math.sqrt(2.0) / float(t), rel=1e-15)


def test_d4_taps_are_orthonormal_daubechies():
    lo, hi, h = G.d4_taps()
    h = np.array(h)
    assert h.sum() == pytest.approx(math.sqrt(2.0))
    assert (h ** 2).sum() == pytest.approx(1.0)
    assert h[0] * h[2] + h[1] * h[3] == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("f,name", FILTERS)
@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("K", [2, 4, 16, 126])
def test_perfect_reconstruction(oracle, f, name, side, K):
    """eq. 11 / 13 and the causal D4 condition P(z)P~'(z^-1) = z^-1 I."""
    v = np.random.default_rng(K).standard_normal(K)
    a, b = oracle.lift_level(f, side, v)
    np.testing.assert_allclose(oracle.lift_level_inv(f, side, a, b), v, rtol=0, atol=1e-13)


@pytest.mark.parametrize("f,name", FILTERS)
@pytest.mark.parametrize("K", [4, 32, 130])
def test_dual_analysis_pairing(oracle, f, name, K):
    """<A u, D v> = <u, v> for primal A and dual D (eq. 13 / 15; eq. 4 at one level)."""
    g = np.random.default_rng(K + f)
    for _ in range(3):
        u = g.standard_normal(K)
        v = g.standard_normal(K)
        a, b = oracle.lift_level(f, 0, u)
        c, d = oracle.lift_level(f, 1, v)
        assert a @ c + b @ d == pytest.approx(u @ v, abs=1e-12 * (np.abs(u) @ np.abs(v)))


def test_d4_energy_equivalence(oracle):
    """Orthogonal filterbank: ||x||^2 = ||a||^2 + ||b||^2 (Sec. II)."""
    v = np.random.default_rng(5).standard_normal(256)
    a, b = oracle.lift_level(0, 0, v)
    assert a @ a + b @ b == pytest.approx(v @ v, rel=1e-14)


@pytest.mark.parametrize("f,side,moments", [(0, 0, 2), (0, 1, 2), (1, 0, 2), (1, 1, 2), (2, 0, 4), (2, 1, 2)])
def test_vanishing_moments(oracle, f, side, moments):
    """Highpass outputs vanish on polynomials below the filter's order.

    Sec. III-B/III-C give two vanishing moments for D4 and 5/3 and four for
    CDF 9/7.  With the rational Table I constants (t = 5/4) the primal (x side)
    highpass keeps four exactly, while the dual (y side) highpass, the
    modulated finite-precision lowpass h~ of Sec. III-C, keeps two exactly and
    only approximately annihilates quadratics and cubics."""
    K = 256
    n = np.arange(K, dtype=np.float64) / K
    for p in range(moments):
        _, b = oracle.lift_level(f, side, n ** p)
        assert np.abs(b[8:K // 2 - 8]).max() < 1e-12, (f, side, p)
    _, b = oracle.lift_level(f, side, n ** moments)
    assert np.abs(b[8:K // 2 - 8]).max() > 1e-9
    if (f, side) == (2, 1):
        _, b = oracle.lift_level(f, side, n ** 2)
        assert np.abs(b[8:K // 2 - 8]).max() < 1e-5


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("K", [2, 8, 64, 1000])
def test_int53_reversible(oracle, side, K):
    v = np.random.default_rng(K + side).integers(-32768, 32768, size=K)
    a, b = oracle.int53_level(side, v)
    np.testing.assert_array_equal(oracle.int53_level_inv(side, a, b), v)


@pytest.mark.parametrize("side", [0, 1])
def test_int53_tracks_float_53(oracle, side):
    """Integer steps differ from the float 5/3 only by the dropped scaling and
    floor rounding (x side: b_int = 2 b; y side: d_int = d / 2)."""
    v = np.random.default_rng(9).integers(-30000, 30000, size=512)
    a, b = oracle.int53_level(side, v)
    af, bf = oracle.lift_level(1, side, v.astype(np.float64))
    np.testing.assert_allclose(a, af, atol=1.0)
    if side == 0:
        np.testing.assert_allclose(b, 2.0 * bf, atol=1.0)
    else:
        np.testing.assert_allclose(b, 0.5 * bf, atol=1.0)


def test_int53_floor_rounding_on_negative_values(oracle):
    """Rounding is floor (toward minus infinity), not truncation."""
    # x side: o' = o - floor((e0 + e1)/2) with e0 + e1 = -3 -> floor(-1.5) = -2
    a, b = oracle.int53_level(0, np.array([-1, 0, -2, 0]))
    assert b[0] == 0 - (-2)
    # y side: e' = e + floor((o[n] + o[n-1] + 1)/2) with o sum = -4 -> floor(-3/2) = -2
    a, b = oracle.int53_level(1, np.array([0, -2, 0, -2]))
    assert a[0] == -2
