"""sidwt_correlate_again: one analysed batch correlated against further stored
signals without analysing it again.  Its full output r and its peaks equal,
bit for bit, those of sidwt_correlate on the same pulses (the same pyramid,
the same kernels), in every precision.  A batch size other than the last
analysis's, a plan that has analysed nothing, and a workspace reallocated
since are refused."""
import numpy as np
import pytest
import torch

from paper_cs_0607001_gb300 import inputs
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

N, J, B = 1024, 4, 150


@pytest.fixture(scope="module")
def batch():
    return inputs.random_batch(n_refs=3, B=B, N=N, J=J, seed=23)


def plan_with_refs(w, filt="cdf97"):
    from paper_cs_0607001_gb300 import sidwt
    p = sidwt.Plan(filt, N, J)
    for x in w["refs"]:
        p.store_reference(U.to_dev_c64(x))
    return p


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "tf32x3"])
def test_again_equals_a_full_call(batch, precision):
    w = batch
    y = U.to_dev_c64(w["y"])
    g = np.random.default_rng(5)
    ids_a = torch.from_numpy(g.integers(0, 3, B).astype(np.int32)).to(U.dev())
    ids_b = torch.from_numpy(g.integers(0, 3, B).astype(np.int32)).to(U.dev())
    with plan_with_refs(w) as p:
        p.correlate(ids_a, y, precision=precision)
        r_again = p.correlate_again(ids_b, precision=precision, want_r=True)
        got = [t.cpu().numpy() for t in p.peaks(B)]
        p.check()
        r_full = p.correlate(ids_b, y, precision=precision, want_r=True)
        want = [t.cpu().numpy() for t in p.peaks(B)]
        p.check()
    np.testing.assert_array_equal(r_again.cpu().numpy(), r_full.cpu().numpy())
    for a, b in zip(got, want):
        np.testing.assert_array_equal(a, b)


def test_again_after_analyze(batch):
    w = batch
    y = U.to_dev_c64(w["y"])
    ids = torch.zeros(B, dtype=torch.int32, device=U.dev())
    with plan_with_refs(w) as p:
        p.analyze_into(y)
        p.correlate_again(ids, precision="bf16x3")
        got = [t.cpu().numpy() for t in p.peaks(B)]
        p.correlate(ids, y, precision="bf16x3")
        want = [t.cpu().numpy() for t in p.peaks(B)]
        p.check()
    for a, b in zip(got, want):
        np.testing.assert_array_equal(a, b)


def test_again_is_refused_without_a_matching_analysis(batch):
    from paper_cs_0607001_gb300 import sidwt
    w = batch
    y = U.to_dev_c64(w["y"])
    ids = torch.zeros(B, dtype=torch.int32, device=U.dev())
    with plan_with_refs(w) as p:
        with pytest.raises(sidwt.SidwtError, match="EINVAL.*last analysis"):
            p.correlate_again(ids)  # nothing analysed yet
        p.correlate(ids, y)
        with pytest.raises(sidwt.SidwtError, match="EINVAL.*last analysis"):
            p.correlate_again(ids[:B - 1].contiguous())  # another batch size
        p.correlate_again(ids[:0].contiguous())  # an empty batch does nothing
        p.reserve(3, 4 * B)  # the workspace is reallocated: the pyramids are gone
        with pytest.raises(sidwt.SidwtError, match="EINVAL.*last analysis"):
            p.correlate_again(ids)


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3"])
def test_again_with_the_same_grouping_reuses_the_packed_operands(batch, precision):
    """The same ids again: the pulses' packed operands are kept (the grouping
    is stable and unchanged), and the result is the first call's, bit for
    bit; then other ids (the grouping changes, so they are packed again) and
    the first ids once more (packed again) give a fresh call's results."""
    w = batch
    y = U.to_dev_c64(w["y"])
    g = np.random.default_rng(8)
    ids_a = torch.from_numpy(g.integers(0, 3, B).astype(np.int32)).to(U.dev())
    ids_b = torch.from_numpy(g.integers(0, 3, B).astype(np.int32)).to(U.dev())

    def fresh(ids):
        with plan_with_refs(w) as q:
            r = q.correlate(ids, y, precision=precision, want_r=True)
            return r.cpu().numpy(), [t.cpu().numpy() for t in q.peaks(B)]

    want_a, want_b = fresh(ids_a), fresh(ids_b)
    with plan_with_refs(w) as p:
        p.correlate(ids_a, y, precision=precision)
        for ids, want in ((ids_a, want_a), (ids_a, want_a), (ids_b, want_b), (ids_a, want_a)):
            r = p.correlate_again(ids, precision=precision, want_r=True)
            got = [t.cpu().numpy() for t in p.peaks(B)]
            np.testing.assert_array_equal(r.cpu().numpy(), want[0])
            for a, b in zip(got, want[1]):
                np.testing.assert_array_equal(a, b)
        p.check()
