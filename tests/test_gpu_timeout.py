"""Failure detection on the device without a GPU fault: a bounded wait that
runs out is recorded, reported on the host, and leaves the context usable.

sidwt_debug_stall makes a wait run out on purpose by never starting what it
waits for (no copy, no MMA is issued, so nothing is left in flight):
  * the pipelined received analysis: sidwt_check then reports SIDWT_ETIMEOUT
    with the analysis named, and the next regular call on the same plan is
    correct again;
  * the tensor-core self-test: its err word gets the timeout bit, and the
    kernel still releases its tensor memory, which the tensor-core correlation
    that follows needs on every SM (an unreleased allocation would block it);
  * the ragged analysis (short pulses on the pipelined kernel, long ones in
    tiles): sidwt_ragged_check reports SIDWT_ETIMEOUT, and the next batch on
    the same object is correct;
  * the serving loop: every request of the batch fails with SIDWT_ETIMEOUT,
    and requests after it are served correctly.
"""
import numpy as np
import pytest
import torch

from paper_cs_0607001_gb300 import inputs
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture
def stall():
    from paper_cs_0607001_gb300 import sidwt
    yield sidwt.debug_stall
    sidwt.debug_stall(0)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_analysis_wait_runs_out_and_is_reported(stall, precision):
    from paper_cs_0607001_gb300 import sidwt
    N, J, B = 1024, 4, 40
    w = inputs.random_batch(n_refs=1, B=B, N=N, J=J, seed=31)
    with sidwt.Plan("cdf97", N, J) as p:
        p.store_reference(U.to_dev_c64(w["refs"][0]))
        ids = torch.zeros(B, dtype=torch.int32, device=U.dev())
        y = U.to_dev_c64(w["y"])
        stall(sidwt.STALL_ANALYSIS)
        p.correlate(ids, y, precision=precision)
        p.peaks(B)
        with pytest.raises(sidwt.SidwtError, match="ETIMEOUT.*received analysis"):
            p.check()
        stall(0)
        p.correlate(ids, y, precision=precision)
        lag, _, _ = p.peaks(B)
        p.check()  # the record was cleared by the failing check; the new call is clean
        assert (lag[:, 0].cpu().numpy() == w["delays"]).all()


def test_tc_selftest_wait_runs_out_and_releases_tensor_memory(stall):
    from paper_cs_0607001_gb300 import sidwt
    from tests.test_gpu_tc import selftest_expected
    stall(sidwt.STALL_TC_SELFTEST)
    _, err = sidwt.tc_selftest()
    torch.cuda.synchronize()
    assert int(err.item()) & 4, "the self-test's bounded wait should have run out"
    stall(0)
    out, err = sidwt.tc_selftest()
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    exp, _, _ = selftest_expected()
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.float64), exp)
    # a tensor-core correlation over every SM allocates tensor memory on each of them
    N, J, B = 2048, 4, 600
    w = inputs.random_batch(n_refs=1, B=B, N=N, J=J, seed=32)
    with sidwt.Plan("legall53", N, J) as p:
        p.store_reference(U.to_dev_c64(w["refs"][0]))
        p.correlate(torch.zeros(B, dtype=torch.int32, device=U.dev()), U.to_dev_c64(w["y"]), precision="bf16x3")
        lag, _, _ = p.peaks(B)
        p.check()
        assert (lag[:, 0].cpu().numpy() == w["delays"]).all()


def ragged_batch(seed):
    """Pulses for both ragged analysis kernels: short ones (the pipelined
    kernel over the item list) and long ones (tiles of 4096 samples plus a
    tail per pulse), each its own reference circularly delayed."""
    g = np.random.default_rng(seed)
    specs = [(1, 1024, 3), (2, 3000, 2), (0, 2048, 4), (2, 20480, 6), (1, 16384, 5), (0, 12288, 3)]
    refs, ys, delays = [], [], []
    for f, N, J in specs:
        x = ((g.standard_normal(N) + 1j * g.standard_normal(N)) / np.sqrt(2)).astype(np.complex64)
        D = int(g.integers(0, N))
        refs.append(x)
        ys.append(np.roll(x, D) + 0.1 * (g.standard_normal(N) + 1j * g.standard_normal(N)))
        delays.append(D)
    offsets = np.concatenate([[0], np.cumsum([s[1] for s in specs])[:-1]]).astype(np.int64)
    return specs, refs, np.concatenate(ys).astype(np.complex64), offsets, delays


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_ragged_analysis_wait_runs_out_and_is_reported(stall, precision):
    from paper_cs_0607001_gb300 import sidwt
    specs, refs, ypack, offsets, delays = ragged_batch(41)
    with sidwt.Ragged() as rg:
        rg.set_precision(precision)
        ids = [rg.store_reference(f, N, J, U.to_dev_c64(x)) for (f, N, J), x in zip(specs, refs)]
        y = U.to_dev_c64(ypack)
        stall(sidwt.STALL_ANALYSIS)
        n = rg.correlate(ids, offsets, y)
        rg.peaks(n)
        with pytest.raises(sidwt.SidwtError, match="ETIMEOUT.*received analysis"):
            rg.check()
        stall(0)
        n = rg.correlate(ids, offsets, y)
        lag, _, _ = rg.peaks(n)
        rg.check()  # the failing check cleared the record; the new call is clean
        first, _ = rg.slots_of(ids)
        lag = lag.cpu().numpy()
        assert [int(lag[s]) for s in first] == delays


def test_serving_batch_whose_wait_runs_out_fails_with_etimeout(stall):
    from paper_cs_0607001_gb300 import sidwt
    from tests.test_gpu_serve import make_requests, new_server, waveforms
    waves = waveforms()
    reqs = make_requests(3, 19, waves)
    with new_server(lanes=1, precision="bf16x3") as srv:
        for w in waves:
            srv.add_waveform(w)
        srv.start()
        stall(sidwt.STALL_ANALYSIS)
        bad = [srv.submit(r["wave"], r["f"], r["N"], r["J"], r["y"]) for r in reqs]
        srv.drain(60.0)  # every request finished (failed ones too)
        for rid in bad:
            with pytest.raises(sidwt.SidwtError, match="ETIMEOUT.*bounded device wait"):
                srv.result(rid)
        stall(0)
        good = [srv.submit(r["wave"], r["f"], r["N"], r["J"], r["y"]) for r in reqs]
        srv.drain(60.0)
        for rid, r in zip(good, reqs):
            lag = srv.result(rid)[0]
            assert int(lag[0]) == r["D"]
