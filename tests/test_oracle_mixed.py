"""Pins of the oracle's mixed-shape batch (pairs of different filter, N and J
packed in one buffer, eq. 20 / 20a per pair).

The mixed call is only bookkeeping around the per-pair correlation: it must
read pair i at its own packed offset and write its J_i + 1 peak records at its
own slot.  Two pins, neither of which goes through the mixed call's packing:

  * every slot equals a separate call on that pair alone, bit for bit;
  * scale 0 of every pair equals the textbook circular cross-correlation
    (numpy FFT): its peak lag is the argmax of |sum_k conj(x[k - D]) y[k]|,
    its magnitude that maximum, and on noiseless echoes the lag is the
    injected delay.

The batch mixes all five filters, lengths that are not powers of two (96,
320, 192) and depths 1..6, and leaves gaps of garbage between the packed
pulses, so that a wrong offset, a slot computed as (J + 1) i, or a filter read
from the wrong pair changes some record.
"""
import numpy as np
import pytest

# (filter, N, J): D4, 5/3, 9/7, integer 5/3, integer 9/7, and repeats with other shapes
SPECS = [(0, 96, 3), (1, 320, 6), (2, 64, 2), (3, 256, 5), (4, 128, 4), (1, 192, 1), (2, 512, 4), (0, 32, 5),
         (3, 96, 5), (2, 320, 3)]
GAP = 5  # garbage samples between packed pulses


def signal(g, f, N):
    if f in (3, 4):
        return (g.integers(-3000, 3000, N) + 1j * g.integers(-3000, 3000, N)).astype(np.complex128)
    return g.standard_normal(N) + 1j * g.standard_normal(N)


def build(seed, noiseless=False):
    g = np.random.default_rng(seed)
    xs, ys, delays, offs = [], [], [], []
    at = 0
    for f, N, J in SPECS:
        x = signal(g, f, N)
        D = int(g.integers(0, N))
        y = np.roll(x, D)
        if not noiseless:
            y = y + 0.3 * signal(g, f, N) if f not in (3, 4) else y + np.round(0.3 * signal(g, f, N))
        xs.append(x)
        ys.append(y)
        delays.append(D)
        offs.append(at)
        at += N + GAP
    xp = 1e6 * (g.standard_normal(at) + 1j * g.standard_normal(at))  # garbage in the gaps
    yp = xp.copy()
    for x, y, o in zip(xs, ys, offs):
        xp[o:o + len(x)] = x
        yp[o:o + len(y)] = y
    return xs, ys, delays, np.array(offs), xp, yp


def circular_xcorr(x, y):
    """r[D] = sum_k conj(x[(k - D) mod N]) y[k] for D = 0..N-1 (x delayed by D)."""
    return np.fft.ifft(np.conj(np.fft.fft(x)) * np.fft.fft(y))


@pytest.mark.parametrize("seed", [1, 2])
def test_mixed_slots_equal_single_pair_calls(oracle, seed):
    xs, ys, _, offs, xp, yp = build(seed)
    fs = [s[0] for s in SPECS]
    Ns = [s[1] for s in SPECS]
    Js = [s[2] for s in SPECS]
    lag, mag, norm, _ = oracle.correlate_mixed(fs, Ns, Js, xp, yp, offs)
    assert lag.shape == (sum(J + 1 for J in Js),)
    slot = 0
    for i, (f, N, J) in enumerate(SPECS):
        l1, m1, n1, _, _ = oracle.correlate_batch(f, xs[i][None], ys[i][None], J)
        np.testing.assert_array_equal(lag[slot:slot + J + 1], l1[0], err_msg=f"pair {i} {SPECS[i]}")
        np.testing.assert_array_equal(mag[slot:slot + J + 1], m1[0], err_msg=f"pair {i} {SPECS[i]}")
        np.testing.assert_array_equal(norm[slot:slot + J + 1], n1[0], err_msg=f"pair {i} {SPECS[i]}")
        slot += J + 1


@pytest.mark.parametrize("noiseless", [False, True])
def test_mixed_scale0_is_the_textbook_cross_correlation(oracle, noiseless):
    xs, ys, delays, offs, xp, yp = build(11, noiseless=noiseless)
    fs = [s[0] for s in SPECS]
    Ns = [s[1] for s in SPECS]
    Js = [s[2] for s in SPECS]
    lag, mag, norm, _ = oracle.correlate_mixed(fs, Ns, Js, xp, yp, offs)
    slot = 0
    for i, (f, N, J) in enumerate(SPECS):
        r = np.abs(circular_xcorr(xs[i], ys[i]))
        top = r.max()
        # the integer filters correlate rounded coefficients: each rounded lifting step moves a
        # coefficient by under one unit, 1e-6 to 2e-5 of the peak on these 12-bit signals (the
        # integer forms themselves are pinned elsewhere; a packing mistake moves the peak by O(1))
        tol = 1e-4 if f in (3, 4) else 1e-9
        assert mag[slot] == pytest.approx(top, rel=tol), (i, SPECS[i])
        # the chosen lag is a maximum (smallest delay among exact ties)
        assert r[lag[slot]] >= top * (1 - 2 * tol), (i, SPECS[i], lag[slot], int(np.argmax(r)))
        if noiseless:
            assert lag[slot] == delays[i], (i, SPECS[i])
        # normalised peak: Cauchy-Schwarz at scale 0 (both energies are |x|^2 and |y|^2 there)
        nx, ny = np.linalg.norm(xs[i]), np.linalg.norm(ys[i])
        assert norm[slot] == pytest.approx(top / (nx * ny), rel=2 * tol)
        assert 0 < norm[slot] <= 1 + 2 * tol
        slot += J + 1
