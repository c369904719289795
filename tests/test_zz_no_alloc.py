"""The allocation-free entry point (sidwt_correlate_static) against the
regular plan-based entry point, through the C ABI.

Callers that cannot allocate device memory (a real-time loop that may not call
cudaMalloc once running, or a host whose device memory belongs to another
allocator) use sidwt_correlate_static, which keeps its intermediates in a
fixed static device array.  Two calls in a row on different inputs must each
give the regular path's peaks within the tolerances of the other parity tests;
the second call also shows that the array's leftover contents do not leak into
a new result.  The file name sorts last so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest
import torch

from paper_cs_0607001_gb300 import inputs

pytestmark = pytest.mark.gpu


def regular_peaks(fname, N, J, x, y):
    from paper_cs_0607001_gb300 import sidwt
    dev = torch.device("cuda", 0)
    with sidwt.Plan(fname, N, J) as p:
        p.store_reference(x)
        ids = torch.zeros(y.shape[0], dtype=torch.int32, device=dev)
        p.correlate(ids, y)
        lag, mag, norm = p.peaks(y.shape[0])
        torch.cuda.synchronize()
        return lag.cpu().numpy(), mag.cpu().numpy(), norm.cpu().numpy()


def static_peaks(fname, N, J, x, y):
    from paper_cs_0607001_gb300 import sidwt
    dev = torch.device("cuda", 0)
    B = y.shape[0]
    lag = torch.full((B, J + 1), -7, dtype=torch.int32, device=dev)
    mag = torch.zeros((B, J + 1), dtype=torch.float32, device=dev)
    norm = torch.zeros((B, J + 1), dtype=torch.float64, device=dev)
    sidwt.correlate_static(fname, N, J, x, y, lag, mag, norm)
    torch.cuda.synchronize()
    return lag.cpu().numpy(), mag.cpu().numpy(), norm.cpu().numpy()


def device_inputs(fname, w, dev, shift=0):
    """The stored signal and the pulses on the device; shift > 0 starts the
    pulse buffer that many samples into a larger allocation (integer pulses:
    shift 2 = 8 bytes, so the buffer is not 16-byte aligned)."""
    if fname.endswith("_int"):
        x = torch.from_numpy(inputs.to_iq16(w["refs"].astype(np.complex128))[0]).to(dev)
        yh = torch.from_numpy(inputs.to_iq16(w["y"].astype(np.complex128)))
    else:
        x = torch.from_numpy(w["refs"][0]).to(dev)
        yh = torch.from_numpy(w["y"])
    if not shift:
        return x, yh.to(dev)
    flat = yh.reshape(-1, *yh.shape[2:])
    buf = torch.zeros((flat.shape[0] + shift, *flat.shape[1:]), dtype=flat.dtype, device=dev)
    buf[shift:] = flat.to(dev)
    return x, buf[shift:].view(yh.shape)


@pytest.mark.parametrize("fname", ["cdf97", "d4", "legall53_int", "cdf97_int"])
def test_static_entry_matches_regular_entry_twice_in_a_row(fname):
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    N, J = 1024, 4
    for call, (B, seed) in enumerate([(150, 21), (70, 22)]):
        w = inputs.random_batch(n_refs=1, B=B, N=N, J=J, seed=seed)
        x, y = device_inputs(fname, w, dev)
        lr, mr, nr = regular_peaks(fname, N, J, x, y)
        ls, ms, ns = static_peaks(fname, N, J, x, y)
        np.testing.assert_array_equal(ls, lr, err_msg=f"call {call}")
        np.testing.assert_allclose(ms, mr, rtol=2e-5, err_msg=f"call {call}")
        np.testing.assert_allclose(ns, nr, rtol=5e-5, atol=1e-6, err_msg=f"call {call}")
        assert (ls[:, 0] == w["delays"]).all()


@pytest.mark.parametrize("fname,N,J,B,shift", [
    ("legall53", 1 << 18, 2, 1, 0),      # too long for shared memory: the per-level analysis
    ("legall53_int", 2048, 3, 90, 2),    # pulses 8 bytes off 16: the shared-memory analysis
])
def test_static_entry_other_analysis_paths(fname, N, J, B, shift):
    dev = torch.device("cuda", 0)
    for call, seed in enumerate([23, 24]):
        w = inputs.random_batch(n_refs=1, B=B, N=N, J=J, seed=seed)
        x, y = device_inputs(fname, w, dev, shift)
        if shift:
            assert y.data_ptr() % 16 == 8
        lr, mr, nr = regular_peaks(fname, N, J, x, y)
        ls, ms, ns = static_peaks(fname, N, J, x, y)
        np.testing.assert_array_equal(ls, lr, err_msg=f"call {call}")
        np.testing.assert_allclose(ms, mr, rtol=2e-5, err_msg=f"call {call}")
        np.testing.assert_allclose(ns, nr, rtol=5e-5, atol=1e-6, err_msg=f"call {call}")
        assert (ls[:, 0] == w["delays"]).all()


def test_static_entry_reports_a_wait_that_ran_out():
    """The static entry point has no sidwt_check: when its analysis gives up on
    a bounded wait (forced with the test hook sidwt_debug_stall), every peak
    record of the call says "no peak"; the next call is correct again."""
    from paper_cs_0607001_gb300 import sidwt
    dev = torch.device("cuda", 0)
    N, J, B = 1024, 4, 50
    w = inputs.random_batch(n_refs=1, B=B, N=N, J=J, seed=25)
    x, y = device_inputs("cdf97", w, dev)
    try:
        sidwt.debug_stall(sidwt.STALL_ANALYSIS)
        ls, ms, ns = static_peaks("cdf97", N, J, x, y)
    finally:
        sidwt.debug_stall(0)
    assert (ls == -1).all() and (ms == 0).all() and (ns == 0).all()
    ls, _, _ = static_peaks("cdf97", N, J, x, y)
    lr, _, _ = regular_peaks("cdf97", N, J, x, y)
    np.testing.assert_array_equal(ls, lr)
    assert (ls[:, 0] == w["delays"]).all()


def test_static_entry_rejects_a_batch_beyond_its_array():
    from paper_cs_0607001_gb300 import sidwt
    dev = torch.device("cuda", 0)
    N, J, B = 8192, 5, 4096
    x = torch.zeros(N, dtype=torch.complex64, device=dev)
    y = torch.zeros((B, N), dtype=torch.complex64, device=dev)
    lag = torch.zeros((B, J + 1), dtype=torch.int32, device=dev)
    mag = torch.zeros((B, J + 1), dtype=torch.float32, device=dev)
    norm = torch.zeros((B, J + 1), dtype=torch.float64, device=dev)
    with pytest.raises(sidwt.SidwtError, match="EINVAL.*static array"):
        sidwt.correlate_static("cdf97", N, J, x, y, lag, mag, norm)
