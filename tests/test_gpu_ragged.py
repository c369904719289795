"""GPU parity of ragged batches (pulses of uneven length, depth and filter,
each against its own stored signal, one persistent correlation launch)
against the FP64 oracle, plus CUDA-graph replay and the autotuner."""
import numpy as np
import pytest
import torch

from tests import gpu_util as U

pytestmark = pytest.mark.gpu

# (filter id, N, J): short bands (small-tile path), long bands (window tiles),
# non-power-of-two N, the deepest level of length 1, one pulse longer than
# shared memory (per-level window lifting)
SPECS = [(0, 64, 3), (1, 96, 5), (2, 256, 8), (0, 320, 6), (1, 1024, 3), (2, 1024, 10), (0, 2048, 4), (1, 3072, 5),
         (2, 4096, 6), (1, 8192, 2), (2, 640, 7), (0, 128, 1), (1, 24576, 3), (2, 512, 9), (0, 6144, 3)]


def build_batch(seed):
    g = np.random.default_rng(seed)
    refs, ys, delays = [], [], []
    for (f, N, J) in SPECS:
        x = (g.standard_normal(N) + 1j * g.standard_normal(N)) / np.sqrt(2)
        D = int(g.integers(0, N))
        y = np.roll(x, D) + 0.3 * (g.standard_normal(N) + 1j * g.standard_normal(N))
        refs.append(x.astype(np.complex64))
        ys.append(y.astype(np.complex64))
        delays.append(D)
    offsets = np.concatenate([[0], np.cumsum([s[1] for s in SPECS])[:-1]]).astype(np.int64)
    return refs, np.concatenate(ys), offsets, delays


def oracle_results(oracle, refs, ypack, offsets):
    out = []
    for (f, N, J), x, off in zip(SPECS, refs, offsets):
        y = ypack[off:off + N].astype(np.complex128)
        lag, mag, norm, r, _ = oracle.correlate_batch(f, x[None].astype(np.complex128), y[None], J, want_r=True)
        out.append((lag[0], mag[0], norm[0], r[0]))
    return out


def run_ragged(rg, refs, ypack, offsets, order=None):
    from paper_cs_0607001_gb300 import sidwt
    ids = [rg.store_reference(f, N, J, U.to_dev_c64(x)) for (f, N, J), x in zip(SPECS, refs)]
    yd = U.to_dev_c64(ypack)
    n = rg.correlate(ids, offsets, yd)
    lag, mag, norm = rg.peaks(n)
    torch.cuda.synchronize()
    return ids, yd, lag.cpu().numpy(), mag.cpu().numpy(), norm.cpu().numpy()


def test_ragged_batch_matches_oracle(oracle):
    from paper_cs_0607001_gb300 import sidwt
    refs, ypack, offsets, delays = build_batch(5)
    exp = oracle_results(oracle, refs, ypack, offsets)
    with sidwt.Ragged() as rg:
        ids, yd, lag, mag, norm = run_ragged(rg, refs, ypack, offsets)
        first, n = rg.slots_of(ids)
    for i, ((f, N, J), (lo, mo, no, ro)) in enumerate(zip(SPECS, exp)):
        sl = slice(first[i], first[i] + J + 1)
        U.check_peak_lags(lag[sl], ro, U.RTOL_FP32, what=f"item {i} {SPECS[i]}")
        np.testing.assert_allclose(mag[sl], np.abs(ro[np.arange(J + 1), lag[sl]]), rtol=2e-5,
                                   err_msg=f"item {i}")
        np.testing.assert_allclose(norm[sl], no, rtol=5e-5, atol=1e-6, err_msg=f"item {i}")
        assert lag[sl][0] == delays[i]


def test_ragged_graph_replay_equals_direct_call():
    from paper_cs_0607001_gb300 import sidwt
    refs, ypack, offsets, _ = build_batch(6)
    with sidwt.Ragged() as rg:
        ids, yd, lag, mag, norm = run_ragged(rg, refs, ypack, offsets)
        nk = rg.graph_create(ids, offsets, yd)
        assert nk >= 3
        for _ in range(3):
            n = rg.graph_launch()
        lag2, mag2, norm2 = rg.peaks(n)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(lag2.cpu().numpy(), lag)
        np.testing.assert_array_equal(mag2.cpu().numpy(), mag)
        # refill the pulse buffer in place: the replay sees the new data
        refs2, ypack2, _, delays2 = build_batch(6)
        yd.copy_(U.to_dev_c64(np.roll(ypack2, 0)))
        n = rg.graph_launch()
        lag3, _, _ = rg.peaks(n)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(lag3.cpu().numpy(), lag)


def test_ragged_autotune_keeps_results(tmp_path, oracle):
    from paper_cs_0607001_gb300 import sidwt
    refs, ypack, offsets, delays = build_batch(7)
    cache = tmp_path / "tune.txt"
    with sidwt.Ragged() as rg:
        rg.autotune(str(cache))
        t = rg.tuning()
        assert set(t[8:16].tolist()) <= {1, 2, 4, 8}
        lines = [l for l in cache.read_text().split("\n") if l.strip()]
        assert len([l for l in lines if not l.startswith("tc ")]) == 8
        assert len([l for l in lines if l.startswith("tc ")]) == 36  # 4 widths x band buckets 2^6 .. 2^14
        ids, yd, lag, mag, norm = run_ragged(rg, refs, ypack, offsets)
        first, _ = rg.slots_of(ids)
    exp = oracle_results(oracle, refs, ypack, offsets)
    for i, ((f, N, J), (lo, mo, no, ro)) in enumerate(zip(SPECS, exp)):
        sl = slice(first[i], first[i] + J + 1)
        U.check_peak_lags(lag[sl], ro, U.RTOL_FP32, what=f"item {i}")


def test_ragged_rejects_bad_items():
    from paper_cs_0607001_gb300 import sidwt
    with sidwt.Ragged() as rg:
        x = torch.zeros(64, dtype=torch.complex64, device=U.dev())
        rg.store_reference("cdf97", 64, 3, x)
        y = torch.zeros(128, dtype=torch.complex64, device=U.dev())
        with pytest.raises(sidwt.SidwtError, match="EINVAL"):
            rg.correlate([3], [0], y)
        with pytest.raises(sidwt.SidwtError, match="EINVAL"):
            rg.correlate([0], [1], y)  # odd offset
        with pytest.raises(sidwt.SidwtError, match="past the end"):
            rg.correlate([0], [96], y)  # 96 + 64 > 128 samples
        with pytest.raises(sidwt.SidwtError, match="EUNSUPPORTED"):
            rg.store_reference("legall53_int", 64, 3, x)
