"""GPU parity of the lifting kernels against the FP64 oracle: the received
(dual-basis) pyramid, the stored signal's SIDWT tree and the FP64 energies,
for every filter, through the C ABI.  The reversible integer 5/3 path must be
bit-exact."""
import numpy as np
import pytest
import torch

from tests import gpu_util as U

pytestmark = pytest.mark.gpu

# (N, J): several CTAs per level, a non-power-of-two N, the deepest level of
# length 1, and one pulse longer than shared memory (per-level window path)
SHAPES = [(64, 3), (96, 5), (1024, 5), (320, 6), (4096, 6), (8192, 5), (32, 5), (32768, 4)]


@pytest.mark.parametrize("fname,fid", list(U.FLOAT_FILTERS.items()))
@pytest.mark.parametrize("N,J", SHAPES)
def test_received_pyramid_matches_oracle(oracle, fname, fid, N, J):
    from paper_cs_0607001_gb300 import sidwt
    B = 3
    g = np.random.default_rng(N + 7 * J + fid)
    y = (g.standard_normal((B, N)) + 1j * g.standard_normal((B, N))).astype(np.complex64)
    with sidwt.Plan(fname, N, J) as p:
        pyr, en = p.analyze(U.to_dev_c64(y))
        torch.cuda.synchronize()
        pyr = pyr.cpu().numpy().astype(np.complex128)
        en = en.cpu().numpy()
    for b in range(B):
        po, eo = oracle.pyramid_y(fid, y[b].astype(np.complex128), J)
        scale = np.abs(po).max()
        assert np.abs(pyr[b] - po).max() <= 2e-6 * scale * J
        np.testing.assert_allclose(en[b], eo, rtol=2e-6 * J)


@pytest.mark.parametrize("fname,fid", list(U.FLOAT_FILTERS.items()))
@pytest.mark.parametrize("N,J", [(64, 3), (96, 5), (1024, 5), (8192, 5), (32, 5)])
def test_reference_tree_matches_oracle(oracle, fname, fid, N, J):
    from paper_cs_0607001_gb300 import sidwt
    g = np.random.default_rng(N + J + 100 * fid)
    x = (g.standard_normal(N) + 1j * g.standard_normal(N)).astype(np.complex64)
    with sidwt.Plan(fname, N, J) as p:
        r0 = p.store_reference(U.to_dev_c64(x))
        r1 = p.store_reference(U.to_dev_c64(x[::-1].copy()))
        assert (r0, r1) == (0, 1) and p.num_refs == 2
        tree, en = p.reference_tree(1)
        torch.cuda.synchronize()
        tree = tree.cpu().numpy().astype(np.complex128)
        en = en.cpu().numpy()
    to, eo = oracle.tree_x(fid, x[::-1].astype(np.complex128), J)
    assert np.abs(tree - to).max() <= 2e-6 * J * np.abs(to).max()
    np.testing.assert_allclose(en, eo, rtol=2e-6 * J)


INT_FILTERS = [("legall53_int", 3), ("cdf97_int", 4)]


@pytest.mark.parametrize("fname,fid", INT_FILTERS)
@pytest.mark.parametrize("N,J", [(64, 3), (96, 5), (8192, 5), (1024, 10), (32768, 4)])
def test_integer_received_pyramid_bit_exact(oracle, fname, fid, N, J):
    from paper_cs_0607001_gb300 import sidwt
    B = 4
    g = np.random.default_rng(N * J)
    y = g.integers(-32768, 32768, size=(B, N, 2)).astype(np.int16)
    with sidwt.Plan(fname, N, J) as p:
        pyr, en = p.analyze(U.to_dev_i16(y))
        torch.cuda.synchronize()
        pyr = pyr.cpu().numpy().astype(np.int64)
        en = en.cpu().numpy()
    for b in range(B):
        po, eo = oracle.pyramid_y(fid, U.iq_to_complex(y[b]), J)
        np.testing.assert_array_equal(pyr[b, :, 0], po.real.astype(np.int64))
        np.testing.assert_array_equal(pyr[b, :, 1], po.imag.astype(np.int64))
        np.testing.assert_allclose(en[b], eo, rtol=1e-12)


@pytest.mark.parametrize("fname,fid", INT_FILTERS)
@pytest.mark.parametrize("N,J", [(64, 3), (96, 5), (8192, 5)])
def test_integer_tree_bit_exact(oracle, fname, fid, N, J):
    from paper_cs_0607001_gb300 import sidwt
    g = np.random.default_rng(N + 3)
    x = g.integers(-32768, 32768, size=(N, 2)).astype(np.int16)
    with sidwt.Plan(fname, N, J) as p:
        p.store_reference(U.to_dev_i16(x))
        tree, en = p.reference_tree(0)
        torch.cuda.synchronize()
        tree = tree.cpu().numpy().astype(np.int64)
        en = en.cpu().numpy()
    to, eo = oracle.tree_x(fid, U.iq_to_complex(x), J)
    np.testing.assert_array_equal(tree[:, 0], to.real.astype(np.int64))
    np.testing.assert_array_equal(tree[:, 1], to.imag.astype(np.int64))
    np.testing.assert_allclose(en, eo, rtol=1e-12)


@pytest.mark.parametrize("fname,fid", INT_FILTERS)
def test_full_size_int16_batch_bit_exact_on_sampled_pulses(oracle, fname, fid):
    """The 4096 x 8192, J = 5 int16 I/Q batch in one call; every coefficient
    of a seeded sample of pulses compared bit for bit."""
    from paper_cs_0607001_gb300 import inputs, sidwt
    w = inputs.two_ref_batch(B=4096, N=8192, J=5)
    yi = inputs.to_iq16(w["y"].astype(np.complex128))
    with sidwt.Plan(fname, 8192, 5) as p:
        pyr, _ = p.analyze(U.to_dev_i16(yi))
        torch.cuda.synchronize()
        sample = [0, 1, 2047, 2048, 3000, 4095]
        got = pyr[sample].cpu().numpy().astype(np.int64)
    for i, b in enumerate(sample):
        po, _ = oracle.pyramid_y(fid, U.iq_to_complex(yi[b]), 5)
        np.testing.assert_array_equal(got[i, :, 0], po.real.astype(np.int64))
        np.testing.assert_array_equal(got[i, :, 1], po.imag.astype(np.int64))
