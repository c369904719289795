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


# Bounds of the split tensor-core products (bf16 hi+lo: u = 2^-16, 16 products
# per MMA; 3xTF32: u = 2^-22, 8 per MMA), per (pair, scale), on
# max_D |r_gpu - r_oracle|.  With a_k the stored coefficients of one variant band
# (advanced by D) and b_k the received ones, each kept product hi*hi + hi*lo +
# lo*hi is off by |e_k| <= 3 u |a_k||b_k| (the dropped lo*lo and the roundings
# of the lo parts); the sums are accumulated in FP32.
#   worst case: (3 u + K 2^-24) max_v ||w_v|| ||u||
#     (FP32 summation of K terms, every rounding at its bound and of one sign;
#     Cauchy-Schwarz over the band);
#   per MMA step: (3 u + s 2^-23) max_v ||w_v|| ||u||, s = 3 ceil(K / k_mma)
#     (the tensor cores add each MMA's products to the running sum in TMEM
#     once; each such step loses at most one unit in the last place of the
#     running sum, whose size is at most sum_k |a_k b_k|).  The loss is a bias,
#     not a random walk: at a matched peak all products have one phase and the
#     measured error grows linearly with K, about half a unit per step (0.42 of
#     this bound on dense random pulses, 0.2 on the LFM / Barker batch, where
#     only the steps that hold the pulse's samples add anything).
def split_bounds(tree, pyr, N, J, j, u, k_mma=None):
    """(worst-case, per-MMA-step) bound for scale j; tree and pyr from the
    oracle (tree_x, pyramid_y); k_mma: products per MMA (16 for bf16, 8 for
    TF32; default from u)."""
    if k_mma is None:
        k_mma = 16 if u >= 2.0 ** -16 else 8
    lev = j + 1 if j < J else J
    Kp = N >> lev
    base = 2 * N * (lev - 1)
    A = tree[base:base + N].reshape(1 << lev, Kp)
    Bb = tree[base + N:base + 2 * N].reshape(1 << lev, Kp)
    off = 2 * N - 4 * Kp
    if j < J:
        wn = np.sqrt((np.abs(A) ** 2).sum(1) + (np.abs(Bb) ** 2).sum(1)).max()
        un = np.linalg.norm(pyr[off:off + 2 * Kp])
        K = 2 * Kp
    else:
        wn = np.sqrt((np.abs(A) ** 2).sum(1)).max()
        un = np.linalg.norm(pyr[off:off + Kp])
        K = Kp
    steps = 3 * -(-K // k_mma)
    worst = (3 * u + K * 2.0 ** -24) * wn * un
    step = (3 * u + steps * 2.0 ** -23) * wn * un
    return worst, step
