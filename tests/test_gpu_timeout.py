"""Failure detection on the device without a GPU fault: a bounded wait that
runs out is recorded, reported on the host, and leaves the context usable.

sidwt_debug_stall makes a wait run out on purpose by never starting what it
waits for (no copy, no MMA is issued, so nothing is left in flight):
  * the pipelined received analysis: sidwt_check then reports SIDWT_ETIMEOUT
    with the analysis named, and the next regular call on the same plan is
    correct again;
  * the tensor-core self-test: its err word gets the timeout bit, and the
    kernel still releases its tensor memory, which the tensor-core correlation
    that follows needs on every SM (an unreleased allocation would block it).
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
