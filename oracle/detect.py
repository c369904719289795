"""Per-scale target detection on the multiresolution correlation (FP64 oracle).

TEST INFRASTRUCTURE ONLY: the CUDA library never imports it.

Sec. V-A (Fig. 6): echoes of several point targets; at each scale the targets
that the scale resolves show as separate peaks of |r_j| above a dB level,
nearby targets merge into one peak at coarser scales.  The paper names no
rule; this build's reading: a detection at scale j is a delay D whose
magnitude is a local maximum along the delay axis (circularly: strictly above
the previous delay, not below the next, so a flat top counts once, at its
first delay) and within `threshold_db` of the scale's largest magnitude.
Detections are reported in increasing delay; at most `max_det` are kept
(the first ones by delay) together with the total count.
"""
from __future__ import annotations

import numpy as np


def detect_row(r: np.ndarray, threshold_db: float) -> np.ndarray:
    """Delays of the detections of one scale (all of them, increasing)."""
    m = np.abs(r)
    top = m.max()
    if top == 0.0:
        return np.zeros(0, np.int64)
    level = top * 10.0 ** (-threshold_db / 20.0)
    prev = np.roll(m, 1)
    nxt = np.roll(m, -1)
    hit = (m > prev) & (m >= nxt) & (m >= level)
    return np.nonzero(hit)[0].astype(np.int64)


def detect(r: np.ndarray, threshold_db: float = 10.0, max_det: int = 32):
    """Per scale of r[j][D]: (count, delays[:max_det], magnitudes[:max_det])."""
    out = []
    for j in range(r.shape[0]):
        d = detect_row(r[j], threshold_db)
        out.append((int(d.shape[0]), d[:max_det], np.abs(r[j][d[:max_det]])))
    return out
