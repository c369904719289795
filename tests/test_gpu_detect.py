"""GPU parity of the per-scale target detection (Sec. V-A, Fig. 6) on
multi-target echoes against the oracle's rule applied to its FP64
correlation."""
import numpy as np
import pytest
import torch

from oracle import detect as Dt
from paper_cs_0607001_gb300 import inputs
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

TOL = 1e-4  # relative to the row's largest |r|: FP32 correlation error plus margin


def check_row(count, lags, mags, r_or, thr, max_det, what):
    m = np.abs(r_or)
    top = m.max()
    level = top * 10 ** (-thr / 20)
    N = m.shape[0]
    prev, nxt = np.roll(m, 1), np.roll(m, -1)
    exact = set(Dt.detect_row(r_or, thr).tolist())
    # clear oracle detections (away from the level and from their neighbours) must be found
    clear = {d for d in exact if m[d] - level > TOL * top and m[d] - prev[d] > TOL * top and
             m[d] - nxt[d] > TOL * top}
    got = set(int(v) for v in lags[:min(count, max_det)])
    if count <= max_det:
        assert clear <= got, f"{what}: missing {sorted(clear - got)}"
    # every reported detection is a local maximum above the level within the tolerance
    for d, g in zip(lags[:min(count, max_det)], mags[:min(count, max_det)]):
        d = int(d)
        assert m[d] >= level - TOL * top and m[d] >= prev[d] - TOL * top and m[d] >= nxt[d] - TOL * top, \
            f"{what}: {d} is not a detection"
        assert abs(g - m[d]) <= TOL * top
    assert abs(count - len(exact)) <= len(exact - clear) + sum(
        1 for d in range(N) if abs(m[d] - level) <= TOL * top or (d not in exact and
                                                                   abs(m[d] - prev[d]) <= TOL * top)), what
    assert list(lags[:min(count, max_det)]) == sorted(lags[:min(count, max_det)])


@pytest.mark.parametrize("thr,N", [(10.0, 2048), (20.0, 2048), (10.0, 32768)])
def test_detections_match_oracle(oracle, thr, N):
    """N = 2048 rows take the shared-memory kernel, N = 32768 the streaming one."""
    from paper_cs_0607001_gb300 import sidwt
    J, B = 4, 6 if N <= 2048 else 2
    w = inputs.multi_target(B=B, N=N, J=J, TB=160, snr_db=20.0, seed=9)
    with sidwt.Plan("cdf97", N, J) as p:
        p.store_reference(U.to_dev_c64(w["refs"][0]))
        ids = torch.zeros(B, dtype=torch.int32, device=U.dev())
        r = p.correlate(ids, U.to_dev_c64(w["y"]), precision="fp32", want_r=True)
        count, lag, mag = sidwt.detect(r, threshold_db=thr, max_det=32)
        count, lag, mag = count.cpu().numpy(), lag.cpu().numpy(), mag.cpu().numpy()
    for b in range(B):
        r_or = oracle.correlate(2, w["refs"][0].astype(np.complex128), w["y"][b].astype(np.complex128), J)
        for j in range(J + 1):
            check_row(int(count[b, j]), lag[b, j], mag[b, j], r_or[j], thr, 32, f"pulse {b} scale {j}")
        # the strongest target is detected at scale 0
        assert int(w["delays"][b]) in set(lag[b, 0][:count[b, 0]].tolist())


def test_detect_edge_cases():
    from paper_cs_0607001_gb300 import sidwt
    r = torch.zeros((3, 16), dtype=torch.complex64, device=U.dev())
    r[1, 0] = 2.0
    r[1, 15] = 1.0
    r[2, 4] = 1.0
    r[2, 5] = 1.0   # flat top: one detection at 4
    r[2, 9] = 1.0
    count, lag, mag = sidwt.detect(r, threshold_db=3.0, max_det=1)
    assert count.cpu().tolist() == [0, 1, 2]
    assert lag.cpu().tolist() == [[-1], [0], [4]]
    with pytest.raises(sidwt.SidwtError, match="EINVAL"):
        sidwt.detect(r, threshold_db=-1.0)
