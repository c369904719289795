"""Coarse-to-fine peak search of the multiresolution correlation (FP64 oracle).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the CUDA library
never imports it.

Sec. V-B: the perfect-reconstruction property lets the coarse scale be
correlated first (at 1/2^J of the input rate), and eq. 21 forms the finer
resolution from the coarser one by inverse lifting; Sec. IV: the peak lag is
the same at every scale (within the scale's own resolution, 2^j samples).
The search this implies (the paper gives no listing; the window rule is this
build's reading): find the peak of scale J over all N delays; then for
j = J-1 down to 0 look only at the delays within w_j = h 2^(j+1) of the
scale-(j+1) peak (circularly) and take the largest |r_j| there, the smallest
delay on ties.  Values come from the oracle's own correlation (eq. 20 / 20a),
so the search only selects among exact values.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def window(center: int, w: int, N: int) -> np.ndarray:
    """Delays within w of center, circularly (all N delays when 2w + 1 >= N)."""
    if 2 * w + 1 >= N:
        return np.arange(N)
    return (center + np.arange(-w, w + 1)) % N


def pick(mag: np.ndarray, cand: np.ndarray) -> int:
    """Largest magnitude among the candidate delays, the smallest delay on ties."""
    m = mag[cand]
    best = m.max()
    return int(cand[m == best].min())


def search(r: np.ndarray, h: int) -> tuple[np.ndarray, np.ndarray]:
    """Coarse-to-fine lags and magnitudes from r[j][D] (j = 0..J)."""
    J = r.shape[0] - 1
    N = r.shape[1]
    mag = np.abs(r)
    lags = np.zeros(J + 1, np.int64)
    lags[J] = pick(mag[J], np.arange(N))
    for j in range(J - 1, -1, -1):
        lags[j] = pick(mag[j], window(int(lags[j + 1]), h << (j + 1), N))
    return lags, mag[np.arange(J + 1), lags]


def coarse_to_fine(filter_id: int, x, y, J: int, h: int = 2) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(lags, magnitudes, full r) of the coarse-to-fine search for one pair."""
    r = O.correlate(filter_id, x, y, J)
    lags, mags = search(r, h)
    return lags, mags, r
