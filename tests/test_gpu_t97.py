"""GPU parity of the CDF 9/7 family over the free parameter t (Sec. III-C
Case II) against the oracle with the same t."""
import numpy as np
import pytest
import torch

from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture
def t97(oracle):
    yield oracle
    oracle.set_cdf97_t(0.0)


@pytest.mark.parametrize("t", [0.85, 0.95, 1.1, 1.5, 1.85])
@pytest.mark.parametrize("B", [40, 5])
def test_family_member_matches_oracle(t97, t, B):
    from paper_cs_0607001_gb300 import sidwt
    N, J = 512, 4
    w = U.small_batch(2, B, N, J, seed=int(t * 100) + B)
    t97.set_cdf97_t(t)
    with sidwt.Plan("cdf97", N, J) as p:
        p.set_cdf97_t(t)
        for x in w["refs"]:
            p.store_reference(U.to_dev_c64(x))
        ids = torch.from_numpy(w["ref_ids"].astype(np.int32)).to(U.dev())
        r = p.correlate(ids, U.to_dev_c64(w["y"]), precision="fp32", want_r=True)
        lag, mag, norm = p.peaks(B)
        r, lag, norm = r.cpu().numpy(), lag.cpu().numpy(), norm.cpu().numpy()
    X = w["refs"][w["ref_ids"]].astype(np.complex128)
    lo, mo, no, ro, _ = t97.correlate_batch(2, X, w["y"].astype(np.complex128), J, want_r=True)
    for b in range(B):
        U.check_r(r[b].astype(np.complex128), ro[b], what=f"t={t} pulse {b}")
        U.check_peak_lags(lag[b], ro[b], U.RTOL_FP32, what=f"t={t} pulse {b}")
        np.testing.assert_allclose(norm[b], no[b], rtol=5e-5, atol=1e-6)


def test_parameter_rules():
    from paper_cs_0607001_gb300 import sidwt
    with sidwt.Plan("legall53", 64, 2) as p:
        with pytest.raises(sidwt.SidwtError, match="EINVAL"):
            p.set_cdf97_t(1.1)
    with sidwt.Plan("cdf97", 64, 2) as p:
        for bad in (0.7, 1.0, 2.0):
            with pytest.raises(sidwt.SidwtError, match="EINVAL"):
                p.set_cdf97_t(bad)
        p.set_cdf97_t(1.1)
        p.store_reference(torch.ones(64, dtype=torch.complex64, device=U.dev()))
        with pytest.raises(sidwt.SidwtError, match="EBUSY"):
            p.set_cdf97_t(1.2)
