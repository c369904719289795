"""The continuous-batching serving loop (sidwt_server_*): results in a mix of
concurrent requests equal the results of the same requests alone, agree with
the oracle, oversized requests are rejected by the memory cap, and waits are
bounded."""
import numpy as np
import pytest
import torch

from paper_cs_0607001_gb300 import inputs

pytestmark = pytest.mark.gpu


def make_requests(n, seed, waves):
    g = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        N = int(g.choice([256, 512, 768, 1024, 2048, 4096]))
        Jmax = 0
        while Jmax < 8 and N % (1 << (Jmax + 1)) == 0:
            Jmax += 1
        J = int(g.integers(1, min(Jmax, 8) + 1))
        f = int(g.integers(0, 3))
        w = int(g.integers(0, len(waves)))
        x = np.zeros(N, np.complex128)
        L = min(len(waves[w]), N)
        x[:L] = waves[w][:L]
        D = int(g.integers(0, N))
        y = np.roll(x, D) + 0.05 * (g.standard_normal(N) + 1j * g.standard_normal(N))
        yt = torch.from_numpy(y.astype(np.complex64)).pin_memory()
        reqs.append({"wave": w, "N": N, "J": J, "f": f, "y": yt, "x": x.astype(np.complex64), "D": D})
    return reqs


def waveforms():
    ws = [inputs.lfm(256, 64), inputs.lfm(512, 200), inputs.barker13(208, 16), inputs.barker13(104, 8)]
    g = np.random.default_rng(3)
    ws.append((g.standard_normal(300) + 1j * g.standard_normal(300)) / np.sqrt(2))
    return [w.astype(np.complex64) for w in ws]


def new_server(**kw):
    from paper_cs_0607001_gb300 import sidwt
    cfg = dict(lanes=3, max_batch=8, max_j=8, memory_cap_bytes=512 << 20, max_lane_samples=1 << 16)
    cfg.update(kw)
    srv = sidwt.Server(**cfg)
    return srv


@pytest.mark.parametrize("precision,rtol", [("fp32", 2e-5), ("bf16x3", 1e-4)])
def test_results_alone_equal_results_in_the_mix(oracle, precision, rtol):
    waves = waveforms()
    reqs = make_requests(40, 11, waves)
    with new_server(precision=precision) as srv:
        for w in waves:
            srv.add_waveform(w)
        srv.start()
        ids = [srv.submit(r["wave"], r["f"], r["N"], r["J"], r["y"]) for r in reqs]
        srv.drain(120.0)
        mixed = [srv.result(i) for i in ids]
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["rejected"] == 0
        assert st["batches"] >= 2 and st["max_batch"] >= 2, st  # requests shared batches
        assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        # each request alone
        for r, m in zip(reqs, mixed):
            rid = srv.submit(r["wave"], r["f"], r["N"], r["J"], r["y"])
            srv.wait(rid, 60.0)
            a = srv.result(rid)
            np.testing.assert_array_equal(a[0], m[0])
            np.testing.assert_allclose(a[1], m[1], rtol=1e-6)
            np.testing.assert_allclose(a[2], m[2], rtol=1e-6)
    # the mix against the oracle on a sample
    for r, m in list(zip(reqs, mixed))[:12]:
        lag, mag, norm, _, _ = oracle.correlate_batch(r["f"], r["x"][None].astype(np.complex128),
                                                      r["y"].numpy()[None].astype(np.complex128), r["J"])
        assert m[0][0] == r["D"] == lag[0, 0]
        np.testing.assert_allclose(m[1], mag[0], rtol=rtol)


def test_oversized_request_is_rejected_and_others_served():
    from paper_cs_0607001_gb300 import sidwt
    waves = waveforms()
    with new_server(memory_cap_bytes=64 << 20, lanes=2) as srv:
        for w in waves:
            srv.add_waveform(w)
        srv.start()
        big = torch.zeros(1 << 18, dtype=torch.complex64).pin_memory()
        small = make_requests(3, 5, waves)
        rid_big = srv.submit(0, "cdf97", 1 << 18, 8, big)  # (32 + 16*8) * 2^18 B > 32 MB lane share
        rids = [srv.submit(r["wave"], r["f"], r["N"], r["J"], r["y"]) for r in small]
        with pytest.raises(sidwt.SidwtError, match="ENOMEM"):
            srv.wait(rid_big, 30.0)
        for rid, r in zip(rids, small):
            srv.wait(rid, 30.0)
            assert srv.result(rid)[0][0] == r["D"]
        assert srv.stats()["rejected"] == 1


def test_waits_are_bounded():
    from paper_cs_0607001_gb300 import sidwt
    waves = waveforms()
    with new_server() as srv:
        srv.add_waveform(waves[0])
        r = make_requests(1, 2, waves[:1])[0]
        rid = srv.submit(0, r["f"], r["N"], r["J"], r["y"])  # server not started: nothing runs it
        with pytest.raises(sidwt.SidwtError, match="ETIMEOUT"):
            srv.wait(rid, 0.2)
        with pytest.raises(sidwt.SidwtError, match="ETIMEOUT"):
            srv.drain(0.2)
        srv.start()
        srv.wait(rid, 30.0)
        assert srv.result(rid)[0][0] == r["D"]


def test_bad_requests_rejected_on_submit():
    from paper_cs_0607001_gb300 import sidwt
    with new_server() as srv:
        srv.add_waveform(waveforms()[0])
        y = torch.zeros(100, dtype=torch.complex64)
        with pytest.raises(sidwt.SidwtError, match="EINVAL"):
            srv.submit(0, "cdf97", 100, 3, y)  # 100 % 8 != 0
        y = torch.zeros(128, dtype=torch.complex64)
        with pytest.raises(sidwt.SidwtError, match="EINVAL"):
            srv.submit(9, "cdf97", 128, 3, y)  # unknown waveform
        with pytest.raises(sidwt.SidwtError, match="EINVAL"):
            srv.submit(0, "legall53_int", 128, 3, y)


def test_long_requests_alone_equal_mix_and_find_their_delays():
    """Requests of the serving workload's long end (N = 2^17, 2^18 and a
    non-power-of-two length, J up to 10) on the tensor-core path: the
    scale-0 peak at the injected delay, and the same results alone and
    mixed with short requests."""
    from paper_cs_0607001_gb300 import sidwt
    waves = waveforms()
    g = np.random.default_rng(21)
    specs = [(1 << 17, 10), (1 << 18, 9), (3 * (1 << 15), 8)]
    longs = []
    for N, J in specs:
        x = np.zeros(N, np.complex128)
        x[:len(waves[0])] = waves[0]
        D = int(g.integers(0, N))
        y = np.roll(x, D) + 0.05 * (g.standard_normal(N) + 1j * g.standard_normal(N))
        longs.append({"N": N, "J": J, "D": D, "y": torch.from_numpy(y.astype(np.complex64)).pin_memory()})
    shorts = make_requests(12, 22, waves)
    with new_server(precision="bf16x3", memory_cap_bytes=4 << 30, max_lane_samples=1 << 20, max_j=10) as srv:
        for wv in waves:
            srv.add_waveform(wv)
        srv.start()
        mix = [srv.submit(0, "cdf97", r["N"], r["J"], r["y"]) for r in longs]
        mix += [srv.submit(r["wave"], r["f"], r["N"], r["J"], r["y"]) for r in shorts]
        srv.drain(300.0)
        got = [srv.result(i) for i in mix[:len(longs)]]
        for r, m in zip(longs, got):
            assert m[0][0] == r["D"]
            rid = srv.submit(0, "cdf97", r["N"], r["J"], r["y"])
            srv.wait(rid, 300.0)
            a = srv.result(rid)
            np.testing.assert_array_equal(a[0], m[0])
            np.testing.assert_allclose(a[1], m[1], rtol=1e-6)


def test_lane_keeps_stored_trees_and_starts_afresh_when_full(oracle):
    """A lane reuses the stored tree of a (waveform, filter, N, J) it already
    holds; once its reserved stores are full it starts afresh.  Results stay
    those of the oracle throughout."""
    waves = waveforms()
    g = np.random.default_rng(17)

    def req(w, f, N, J):
        x = np.zeros(N, np.complex128)
        L = min(len(waves[w]), N)
        x[:L] = waves[w][:L]
        D = int(g.integers(0, N))
        y = np.roll(x, D) + 0.05 * (g.standard_normal(N) + 1j * g.standard_normal(N))
        return {"wave": w, "f": f, "N": N, "J": J, "D": D, "x": x,
                "y": torch.from_numpy(y.astype(np.complex64)).pin_memory()}

    few = [req(w, f, 1024, 3) for w, f in [(0, 0), (1, 1), (2, 2)]]
    # 5 waves x 3 filters x 3 (N, J): 45 distinct keys, far more than one
    # lane's stores hold (2 * max_j * max_lane_samples elements)
    many = [req(w, f, N, J) for w in range(5) for f in range(3) for (N, J) in [(1024, 3), (2048, 4), (512, 2)]]
    with new_server(lanes=1, max_batch=4, max_j=4, max_lane_samples=8192) as srv:
        for w in waves:
            srv.add_waveform(w)
        srv.start()
        seq = few * 4 + many + few
        out = []
        for r in seq:
            rid = srv.submit(r["wave"], r["f"], r["N"], r["J"], r["y"])
            srv.wait(rid, 60.0)
            out.append(srv.result(rid))
        st = srv.stats()
    assert st["completed"] == len(seq)
    assert st["ref_hits"] + st["ref_stores"] == len(seq)
    assert st["ref_hits"] >= 9, st  # the repeats of the first three keys
    assert st["ref_stores"] >= len(many) + 3, st  # every distinct key built at least once
    for r, m in zip(seq, out):
        lag, mag, _, _, _ = oracle.correlate_batch(r["f"], r["x"][None], r["y"].numpy()[None].astype(np.complex128),
                                                   r["J"])
        assert m[0][0] == r["D"] == lag[0, 0]
        np.testing.assert_allclose(m[1], mag[0], rtol=2e-5)
