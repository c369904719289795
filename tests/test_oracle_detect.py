"""Pins of the per-scale detection rule (oracle/detect.py)."""
import numpy as np

from oracle import detect as Dt
from paper_cs_0607001_gb300 import inputs


def test_local_maxima_threshold_plateau_and_wrap():
    m = np.zeros(32)
    m[0] = 10.0     # maximum at delay 0: its previous delay is 31 (circular)
    m[31] = 9.0
    m[5] = 4.0      # 20 log10(4/10) = -8 dB: detected at a 10 dB threshold
    m[9] = 3.0      # -10.5 dB: not detected
    m[15] = m[16] = 5.0   # flat top: counted once, at its first delay
    m[20] = 6.0
    m[21] = 7.0     # rising edge: only 21 is a maximum
    got = Dt.detect_row(m.astype(complex), 10.0)
    assert got.tolist() == [0, 5, 15, 21]
    assert Dt.detect_row(m.astype(complex), 5.0).tolist() == [0, 21]  # 5 is -6 dB, 7 is -3.1 dB
    assert Dt.detect_row(np.zeros(8, complex), 10.0).tolist() == []


def test_max_det_keeps_the_first_delays_and_the_count():
    m = np.tile([0.0, 1.0], 8).astype(complex)   # 8 equal maxima
    (cnt, d, mag), = Dt.detect(m[None], 1.0, max_det=3)
    assert cnt == 8 and d.tolist() == [1, 3, 5] and mag.tolist() == [1.0, 1.0, 1.0]


def test_two_separated_targets_found_at_scale_0(oracle):
    """Two LFM echoes 300 samples apart (equal strength, no noise): exactly
    two scale-0 detections, at the two delays (LFM sidelobes sit 13 dB down)."""
    N, J = 2048, 3
    x = inputs.lfm(N, 160)
    y = np.roll(x, 500) + 0.9j * np.roll(x, 800)
    r = oracle.correlate(2, x, y, J)
    cnt, d, _ = Dt.detect(r, 10.0)[0]
    assert cnt == 2 and d.tolist() == [500, 800]


def test_adjacent_targets_merge_at_coarse_scales(oracle):
    """Two echoes one sample apart are one detection from scale 2 on."""
    N, J = 2048, 4
    x = inputs.lfm(N, 160)
    y = np.roll(x, 1000) + np.roll(x, 1001)
    r = oracle.correlate(2, x, y, J)
    det = Dt.detect(r, 10.0)
    for j in range(2, J + 1):
        cnt, d, _ = det[j]
        near = [int(v) for v in d if min(abs(int(v) - 1000), N - abs(int(v) - 1000)) <= 2 << j]
        assert len(near) == 1, (j, d)
