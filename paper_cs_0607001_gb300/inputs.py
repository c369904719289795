"""Seeded synthetic radar workloads (stored pulses and received echoes).

This module only draws inputs; it holds none of the correlation method's
arithmetic.  The same bytes feed the CUDA library and the CPU oracle.

Signals (Sec. IV, eq. 18 and Sec. V-A):
  * LFM chirp of time-bandwidth product Np sampled at the bandwidth:
    x[n] = exp(i*pi*(n - Np/2)^2 / Np) for n < Np, zero-padded to N
    (the "p" of eq. 18 read as pi).
  * Barker-13 phase code (+ + + + + - - + + - + - +), `spc` samples per chip,
    zero-padded to N.  The paper names no phase code; this one stands in for
    the "phase-coded" pulses of the workloads.
  * Received: y = x delayed circularly by D plus complex white Gaussian noise
    of variance P / 10^(SNR/10), P = mean |x|^2 over the pulse's own samples.

Random numbers come from numpy's counter-based Philox generator keyed by
(workload id, purpose), so every draw is reproducible on any machine.
"""
from __future__ import annotations

import numpy as np

BARKER13 = np.array([1, 1, 1, 1, 1, -1, -1, 1, 1, -1, 1, -1, 1], dtype=np.float64)


def rng(workload: int, purpose: int = 0) -> np.random.Generator:
    key = ((workload & 0xFFFFFFFF) << 32) | (purpose & 0xFFFFFFFF)
    return np.random.Generator(np.random.Philox(key=key))


def lfm(N: int, Np: int) -> np.ndarray:
    """Complex LFM chirp of Np samples zero-padded to N (complex128)."""
    Np = int(min(Np, N))
    n = np.arange(Np, dtype=np.float64)
    x = np.zeros(N, np.complex128)
    x[:Np] = np.exp(1j * np.pi * (n - Np / 2.0) ** 2 / Np)
    return x


def barker13(N: int, spc: int) -> np.ndarray:
    """Barker-13 phase code, `spc` samples per chip, zero-padded to N."""
    chips = np.repeat(BARKER13, int(spc))[:N]
    x = np.zeros(N, np.complex128)
    x[:chips.shape[0]] = chips
    return x


def pulse_power(x: np.ndarray) -> float:
    nz = np.abs(x) > 0
    return float(np.mean(np.abs(x[nz]) ** 2)) if nz.any() else 0.0


def echo(x: np.ndarray, delays: np.ndarray, snr_db: np.ndarray, g: np.random.Generator) -> np.ndarray:
    """Received pulses [B][N]: x circularly delayed by delays[b] plus noise at snr_db[b]."""
    B = delays.shape[0]
    N = x.shape[-1]
    X = np.broadcast_to(x, (B, N)) if x.ndim == 1 else x
    n = np.arange(N)
    idx = (n[None, :] - delays[:, None]) % N
    y = np.take_along_axis(np.asarray(X), idx, axis=1)
    P = np.array([pulse_power(X[b]) for b in range(B)]) if x.ndim == 2 else np.full(B, pulse_power(x))
    sigma = np.sqrt(P / 10.0 ** (np.asarray(snr_db, np.float64) / 10.0) / 2.0)
    w = g.standard_normal((B, N)) + 1j * g.standard_normal((B, N))
    return y + sigma[:, None] * w


def to_c64(a: np.ndarray) -> np.ndarray:
    """Round once to complex64 (the bytes both sides receive)."""
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex64))


def to_iq16(a: np.ndarray, peak: float = 0.9 * 32767.0) -> np.ndarray:
    """Scale each row to the given peak and round half to even into int16 I/Q pairs [.., N, 2]."""
    a = np.atleast_2d(a)
    m = np.maximum(np.abs(a.real).max(axis=1), np.abs(a.imag).max(axis=1))
    s = np.where(m > 0, peak / np.where(m > 0, m, 1.0), 1.0)
    re = np.round(a.real * s[:, None])
    im = np.round(a.imag * s[:, None])
    out = np.stack([re, im], axis=-1).astype(np.int16)
    return np.ascontiguousarray(out)


# --------------------------------------------------------------------------
# Workloads.  Each returns a dict with the stored pulses (refs), the received
# pulses (y), the reference index of every received pulse and the drawn
# delays / SNRs, all as numpy arrays.
# --------------------------------------------------------------------------

def single_lfm(N: int = 1024, J: int = 3, TB: int = 64, snr_db: float = 10.0, seed: int = 1):
    """One LFM pulse (TB samples) and one noisy echo with a seeded delay."""
    g = rng(seed, 1)
    x = lfm(N, TB)
    D = np.array([int(g.integers(0, N))])
    y = echo(x, D, np.array([snr_db]), g)
    return {"refs": to_c64(x[None, :]), "y": to_c64(y), "ref_ids": np.zeros(1, np.int32), "delays": D,
            "snr_db": np.array([snr_db]), "N": N, "J": J}


def two_ref_batch(B: int = 4096, N: int = 8192, J: int = 5, TB: int = 256, spc: int = 16, seed: int = 2,
                  snr_lo: float = 0.0, snr_hi: float = 20.0):
    """First half of the batch echoes an LFM pulse (TB samples), second half a
    Barker-13 pulse (spc samples per chip); delays uniform, SNR uniform."""
    g = rng(seed, 2)
    refs = np.stack([lfm(N, TB), barker13(N, spc)])
    ref_ids = (np.arange(B) >= B // 2).astype(np.int32)
    D = g.integers(0, N, size=B)
    snr = g.uniform(snr_lo, snr_hi, size=B)
    y = np.empty((B, N), np.complex128)
    for r in (0, 1):
        sel = ref_ids == r
        y[sel] = echo(refs[r], D[sel], snr[sel], g)
    return {"refs": to_c64(refs), "y": to_c64(y), "ref_ids": ref_ids, "delays": D, "snr_db": snr, "N": N, "J": J}


def many_ref_batch(n_refs: int = 64, B: int = 16384, N: int = 4096, J: int = 6, seed: int = 3):
    """n_refs stored pulses: half LFM with TB log-spaced in [64, 2048], half
    Barker-13 with 1..32 samples per chip; pulse i echoes reference i mod n_refs."""
    g = rng(seed, 3)
    half = n_refs // 2
    tbs = np.unique(np.round(np.logspace(np.log2(64), np.log2(2048), half, base=2.0)).astype(int))
    tbs = np.resize(tbs, half)
    spcs = np.resize(np.arange(1, 33), n_refs - half)
    refs = [lfm(N, int(t)) for t in tbs] + [barker13(N, int(s)) for s in spcs]
    refs = np.stack(refs)
    ref_ids = (np.arange(B) % n_refs).astype(np.int32)
    D = g.integers(0, N, size=B)
    snr = g.uniform(0.0, 20.0, size=B)
    y = echo(refs[ref_ids], D, snr, g)
    return {"refs": to_c64(refs), "y": to_c64(y), "ref_ids": ref_ids, "delays": D, "snr_db": snr, "N": N, "J": J}


def random_batch(n_refs: int, B: int, N: int, J: int, seed: int):
    """Small mixed batch for parity tests: random complex references (unit
    variance) and noisy delayed echoes, pulses assigned to references at random."""
    g = rng(seed, 4)
    refs = (g.standard_normal((n_refs, N)) + 1j * g.standard_normal((n_refs, N))) / np.sqrt(2.0)
    ref_ids = g.integers(0, n_refs, size=B).astype(np.int32)
    D = g.integers(0, N, size=B)
    snr = g.uniform(0.0, 20.0, size=B)
    y = echo(refs[ref_ids], D, snr, g)
    return {"refs": to_c64(refs), "y": to_c64(y), "ref_ids": ref_ids, "delays": D, "snr_db": snr, "N": N, "J": J}


def ragged_batch(n: int = 10000, seed: int = 4, n_lo: int = 256, n_hi: int = 65536, j_lo: int = 3, j_hi: int = 8):
    """n pulses of uneven length: N log-uniform in [n_lo, n_hi] rounded to a
    multiple of 2^J (at least 2^J), J uniform in [j_lo, j_hi], filter uniform
    over the float filters (0 D4, 1 LeGall 5/3, 2 CDF 9/7); half LFM chirps
    (TB = N/8 clamped to [16, 4096]), half Barker-13 codes (samples per chip
    so that the code spans about N/8); delays uniform, SNR uniform in
    0-20 dB.  Each pulse has its own stored reference.  Returns packed
    complex64 arrays (refs, y) with per-item offsets."""
    g = rng(seed, 5)
    J = g.integers(j_lo, j_hi + 1, size=n)
    raw = np.exp(g.uniform(np.log(n_lo), np.log(n_hi), size=n))
    N = np.maximum(np.round(raw / (1 << J)).astype(np.int64), 1) * (1 << J)
    filt = g.integers(0, 3, size=n)
    kind = g.integers(0, 2, size=n)
    D = (g.uniform(0, 1, size=n) * N).astype(np.int64)
    snr = g.uniform(0.0, 20.0, size=n)
    off = np.concatenate([[0], np.cumsum(N)[:-1]]).astype(np.int64)
    tot = int(N.sum())
    refs = np.empty(tot, np.complex64)
    ys = np.empty(tot, np.complex64)
    for i in range(n):
        Ni = int(N[i])
        tb = int(min(max(Ni // 8, 16), 4096, Ni))
        x = lfm(Ni, tb) if kind[i] == 0 else barker13(Ni, max(1, tb // 13))
        y = echo(x, D[i:i + 1], snr[i:i + 1], g)[0]
        refs[off[i]:off[i] + Ni] = x
        ys[off[i]:off[i] + Ni] = y
    return {"refs": refs, "y": ys, "offsets": off, "N": N, "J": J.astype(np.int64), "filter": filt,
            "delays": D, "snr_db": snr}


# Point-target offsets (samples) and reflectivity magnitudes of the
# multi-target echoes: a pair one sample apart, two more targets a few
# samples away, a fifth one further off (Sec. V-A, Fig. 6 narrative).
MT_OFFSETS = np.array([0, 1, 5, 9, -16])
MT_GAINS = np.array([1.0, 0.8, 0.9, 0.7, 0.6])


def multi_target(B: int = 4096, N: int = 8192, J: int = 5, TB: int = 160, snr_db: float = 20.0, seed: int = 6):
    """Echoes of five point targets per pulse (Sec. V-A): y = sum_k s_k x
    delayed by D0 + offset_k, plus noise at snr_db relative to the strongest
    echo; x an LFM chirp with time-bandwidth product TB; D0 uniform, the
    reflectivities' phases uniform."""
    g = rng(seed, 6)
    x = lfm(N, TB)
    D0 = g.integers(0, N, size=B)
    ph = np.exp(2j * np.pi * g.uniform(0, 1, size=(B, MT_OFFSETS.shape[0])))
    n = np.arange(N)
    y = np.zeros((B, N), np.complex128)
    for k in range(MT_OFFSETS.shape[0]):
        idx = (n[None, :] - (D0[:, None] + MT_OFFSETS[k])) % N
        y += (MT_GAINS[k] * ph[:, k])[:, None] * x[idx]
    sigma = np.sqrt(pulse_power(x) / 10.0 ** (snr_db / 10.0) / 2.0)
    y += sigma * (g.standard_normal((B, N)) + 1j * g.standard_normal((B, N)))
    return {"refs": to_c64(x[None, :]), "y": to_c64(y), "ref_ids": np.zeros(B, np.int32), "delays": D0,
            "offsets": MT_OFFSETS, "N": N, "J": J}
