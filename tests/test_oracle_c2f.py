"""Pins of the coarse-to-fine search (oracle/coarse_to_fine.py) and of the
synthesis step it rests on (eq. 21: one level of inverse y-side lifting)."""
import numpy as np
import pytest

from oracle import coarse_to_fine as C
from paper_cs_0607001_gb300 import inputs


def test_window_is_circular_and_saturates():
    assert C.window(1, 2, 16).tolist() == [15, 0, 1, 2, 3]
    assert C.window(15, 1, 16).tolist() == [14, 15, 0]
    assert sorted(C.window(3, 8, 16).tolist()) == list(range(16))


def test_search_keeps_to_the_window_and_breaks_ties_low():
    # scale 2 peaks at 40; scale 1 has its global maximum far away (200) and a
    # smaller local maximum inside the window around 40: the search must
    # take the one inside the window
    N = 256
    r = np.zeros((3, N), complex)
    r[2, 40] = 5.0
    r[1, 200] = 9.0
    r[1, 43] = 4.0
    r[0, 42] = 3.0
    r[0, 44] = 3.0  # tie inside the window: the smaller delay wins
    lags, mags = C.search(r, h=1)   # windows: scale 1 +-4, scale 0 +-2
    assert lags.tolist() == [42, 43, 40]
    assert mags.tolist() == [3.0, 4.0, 5.0]


@pytest.mark.parametrize("fid", [0, 1, 2])
def test_full_windows_equal_full_argmax(oracle, fid):
    """With windows covering every delay the search is the plain per-scale argmax."""
    g = np.random.default_rng(7 + fid)
    N, J = 128, 3
    x = g.standard_normal(N) + 1j * g.standard_normal(N)
    y = np.roll(x, 37) + 0.5 * (g.standard_normal(N) + 1j * g.standard_normal(N))
    lags, mags, r = C.coarse_to_fine(fid, x, y, J, h=N)
    np.testing.assert_array_equal(lags, np.argmax(np.abs(r), axis=1))


@pytest.mark.parametrize("fid", [0, 1, 2])
def test_injected_delay_found_from_the_coarse_scale(oracle, fid):
    """Noiseless LFM echo: the smallest windows (h = 2) still land on the
    injected delay at scale 0 (the peak moves at most 2^j per scale, Sec. IV)."""
    N, J = 1024, 5
    x = inputs.lfm(N, 128)
    for D in (0, 5, 517, 1023):
        lags, _, r = C.coarse_to_fine(fid, x, np.roll(x, D), J, h=2)
        assert lags[0] == D
        assert lags[0] == int(np.argmax(np.abs(r[0])))


@pytest.mark.parametrize("fid", [0, 1, 2])
def test_synthesis_inverts_the_received_analysis(oracle, fid):
    """Eq. 21: one level of inverse y-side lifting rebuilds c_{l-1} from
    (c_l, d_l) of the received pyramid (perfect reconstruction)."""
    g = np.random.default_rng(11)
    N, J = 256, 4
    y = g.standard_normal(N) + 1j * g.standard_normal(N)
    pyr, _ = oracle.pyramid_y(fid, y, J)
    prev = y
    for l in range(1, J + 1):
        H = N >> l
        off = 2 * N - 4 * H
        c, d = pyr[off:off + H], pyr[off + H:off + 2 * H]
        re = oracle.lift_level_inv(fid, 1, c.real, d.real)
        im = oracle.lift_level_inv(fid, 1, c.imag, d.imag)
        np.testing.assert_allclose(re + 1j * im, prev, atol=1e-12)
        prev = c
