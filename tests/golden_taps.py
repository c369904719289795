"""Reads tests/golden/filters.json (the printed filters of Sec. III) into floats."""
import json
import math
import os
from fractions import Fraction

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "filters.json")
_SCALES = {"1": 1.0, "2": 2.0, "1/sqrt2": 1.0 / math.sqrt(2.0), "sqrt2": math.sqrt(2.0)}


def load():
    with open(_PATH) as f:
        return json.load(f)


def taps(entry):
    s = _SCALES[entry["scale"]]
    return {int(k): float(Fraction(v)) * s for k, v in entry["taps"].items()}


def modulated_highpass(lo_unscaled, scale=1.0):
    """Eq. 7 reading: hi[1+m] = (-1)^m lo[m] (times the side's synthesis scaling)."""
    return {1 + m: ((-1) ** abs(m)) * v * scale for m, v in lo_unscaled.items()}


def d4_taps():
    g = load()["d4"]
    h = [(p + q * math.sqrt(3.0)) / (4.0 * math.sqrt(2.0)) for p, q in g["h"]]
    lo = {int(k): h[i] for k, i in g["x_lo_offsets"].items()}
    hi = {int(k): s * h[i] for k, (s, i) in g["x_hi_terms"].items()}
    return lo, hi, h


def filter_taps(name, side):
    """(lo, hi) taps for name in {'legall53', 'cdf97', 'd4'} and side in {'x', 'y'}."""
    g = load()
    if name == "d4":
        lo, hi, _ = d4_taps()
        return lo, hi
    f = g[name]
    if name == "legall53":
        return taps(f[side + "_lo"]), taps(f[side + "_hi"])
    x_lo = taps(f["x_lo"])
    y_lo = taps(f["y_lo"])
    if side == "x":
        return x_lo, modulated_highpass(y_lo)
    return y_lo, modulated_highpass(x_lo)
