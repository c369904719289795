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


@pytest.mark.parametrize("fname", ["cdf97", "d4", "legall53_int"])
def test_static_entry_matches_regular_entry_twice_in_a_row(fname):
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    N, J = 1024, 4
    for call, (B, seed) in enumerate([(150, 21), (70, 22)]):
        w = inputs.random_batch(n_refs=1, B=B, N=N, J=J, seed=seed)
        if fname == "legall53_int":
            x = torch.from_numpy(inputs.to_iq16(w["refs"].astype(np.complex128))[0]).to(dev)
            y = torch.from_numpy(inputs.to_iq16(w["y"].astype(np.complex128))).to(dev)
        else:
            x = torch.from_numpy(w["refs"][0]).to(dev)
            y = torch.from_numpy(w["y"]).to(dev)
        lr, mr, nr = regular_peaks(fname, N, J, x, y)
        ls, ms, ns = static_peaks(fname, N, J, x, y)
        np.testing.assert_array_equal(ls, lr, err_msg=f"call {call}")
        np.testing.assert_allclose(ms, mr, rtol=2e-5, err_msg=f"call {call}")
        np.testing.assert_allclose(ns, nr, rtol=5e-5, atol=1e-6, err_msg=f"call {call}")
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
