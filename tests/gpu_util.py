"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np
import torch

from paper_cs_0607001_gb300 import inputs

FLOAT_FILTERS = {"d4": 0, "legall53": 1, "cdf97": 2}

# FP32 correlation tolerance (per pair and scale, relative to the oracle's
# largest |r|): max_D |r_gpu - r_oracle| <= RTOL_FP32 * max_D |r_oracle|.
RTOL_FP32 = 1e-5


def dev():
    return torch.device("cuda", 0)


def to_dev_c64(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).to(dev())


def to_dev_i16(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.int16))).to(dev())


def iq_to_complex(a: np.ndarray) -> np.ndarray:
    a = a.astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def check_r(r_gpu: np.ndarray, r_or: np.ndarray, rtol=RTOL_FP32, what=""):
    """Per-scale max error relative to the oracle's max |r|; returns the worst ratio."""
    worst = 0.0
    for j in range(r_or.shape[0]):
        scale = np.abs(r_or[j]).max()
        err = np.abs(r_gpu[j] - r_or[j]).max()
        ratio = err / scale if scale > 0 else err
        worst = max(worst, ratio)
        assert ratio <= rtol, f"{what} scale {j}: max err {err:.3e} vs max|r| {scale:.3e} (ratio {ratio:.2e})"
    return worst


def check_peak_lags(lag_gpu: np.ndarray, r_or: np.ndarray, bound: float, what=""):
    """Peak lag per scale: exact when the oracle's top-2 margin exceeds 4x the
    error bound, otherwise any lag whose oracle magnitude is within the bound
    of the maximum (several lags are then correct)."""
    for j in range(r_or.shape[0]):
        m = np.abs(r_or[j])
        top = m.max()
        order = np.argsort(-m, kind="stable")
        second = m[order[1]] if m.shape[0] > 1 else 0.0
        margin = (top - second) / top if top > 0 else 0.0
        g = int(lag_gpu[j])
        if margin > 4 * bound:
            assert g == int(np.argmax(m)), f"{what} scale {j}: lag {g} != oracle {int(np.argmax(m))}"
        else:
            assert 0 <= g < m.shape[0] and m[g] >= top * (1 - 2 * bound), f"{what} scale {j}: lag {g} not a maximum"


def small_batch(n_refs, B, N, J, seed):
    return inputs.random_batch(n_refs=n_refs, B=B, N=N, J=J, seed=seed)
