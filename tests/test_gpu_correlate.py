"""GPU parity of the all-lag, all-scale correlation and its peaks against the
FP64 oracle (eq. 20 / 20a), through the C ABI, plain FP32 path.

Small cases span several pulse tiles (64 pulses), several lag tiles (128 lags)
and ragged tails; the full-size cases run the benchmark's own launch shape and
compare a seeded sample of pulses."""
import numpy as np
import pytest
import torch

from paper_cs_0607001_gb300 import inputs
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def run_plan(fname, N, J, refs, y, ref_ids, precision="fp32", want_r=True):
    from paper_cs_0607001_gb300 import sidwt
    p = sidwt.Plan(fname, N, J)
    is_int = fname in ("legall53_int", "cdf97_int")
    for x in refs:
        p.store_reference(U.to_dev_i16(x) if is_int else U.to_dev_c64(x))
    yd = U.to_dev_i16(y) if is_int else U.to_dev_c64(y)
    ids = torch.from_numpy(ref_ids.astype(np.int32)).to(U.dev())
    r = p.correlate(ids, yd, precision=precision, want_r=want_r)
    lag, mag, norm = p.peaks(y.shape[0])
    torch.cuda.synchronize()
    out = (Rows(r), lag.cpu().numpy(), mag.cpu().numpy(), norm.cpu().numpy())
    p.close()
    return out


class Rows:
    """r[b] rows copied to the host on demand (the full output can be GBs)."""

    def __init__(self, r):
        self.r = r

    def __getitem__(self, b):
        return self.r[int(b)].cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("fname,fid", list(U.FLOAT_FILTERS.items()))
# batches of at most 16 pulses take the latency kernel: (2048, 3, 9) stages
# its scale-0 bands in two chunks of the received band, (8192, 5, 3) reads
# scale 0's bands (too long to stage) straight from memory
@pytest.mark.parametrize("N,J,B,nrefs", [(1024, 4, 150, 3), (96, 5, 70, 2), (320, 6, 9, 1), (2048, 3, 65, 1),
                                         (64, 6, 5, 4), (16, 1, 40, 2), (2, 1, 3, 1), (2048, 3, 9, 2),
                                         (8192, 5, 3, 1)])
def test_correlation_matches_oracle(oracle, fname, fid, N, J, B, nrefs):
    w = U.small_batch(nrefs, B, N, J, seed=N + B + fid)
    r, lag, mag, norm = run_plan(fname, N, J, w["refs"], w["y"], w["ref_ids"])
    X = w["refs"][w["ref_ids"]].astype(np.complex128)
    Y = w["y"].astype(np.complex128)
    lo, mo, no, ro, _ = oracle.correlate_batch(fid, X, Y, J, form=1, want_r=True)
    ex = [oracle.tree_x(fid, x.astype(np.complex128), J)[1] for x in w["refs"]]
    for b in range(B):
        U.check_r(r[b], ro[b], what=f"{fname} pulse {b}")
        U.check_peak_lags(lag[b], ro[b], U.RTOL_FP32, what=f"{fname} pulse {b}")
        np.testing.assert_allclose(mag[b], np.abs(ro[b][np.arange(J + 1), lag[b]]), rtol=2e-5)
        np.testing.assert_allclose(norm[b], no[b], rtol=5e-5, atol=1e-6)
        # the normalisation alone: the GPU's |r| at its lag over the oracle's FP64
        # energies (eq. 1), so that only the GPU energies' error is left, held to
        # the energies' own tolerance (2e-6 J, as in the lifting tests)
        ey = oracle.pyramid_y(fid, Y[b], J)[1]
        for j in range(J + 1):
            D = int(lag[b][j])
            e_x = ex[w["ref_ids"][b]][(1 << j) - 1 + (D & ((1 << j) - 1))]
            want = float(mag[b][j]) / np.sqrt(e_x * ey[j])
            assert abs(norm[b][j] - want) <= 2e-6 * J * want + 1e-12, (b, j, norm[b][j], want)


@pytest.mark.parametrize("fname,fid", [("legall53_int", 3), ("cdf97_int", 4)])
@pytest.mark.parametrize("B", [70, 6])
def test_integer_plan_correlation_matches_oracle(oracle, fname, fid, B):
    N, J = 512, 4
    w = inputs.random_batch(n_refs=2, B=B, N=N, J=J, seed=9)
    refs = inputs.to_iq16(w["refs"].astype(np.complex128))
    y = inputs.to_iq16(w["y"].astype(np.complex128))
    r, lag, mag, norm = run_plan(fname, N, J, refs, y, w["ref_ids"])
    X = U.iq_to_complex(refs[w["ref_ids"]])
    Y = U.iq_to_complex(y)
    _, _, no, ro, _ = oracle.correlate_batch(fid, X, Y, J, form=1, want_r=True)
    for b in range(B):
        U.check_r(r[b], ro[b], what=f"int pulse {b}")
        U.check_peak_lags(lag[b], ro[b], U.RTOL_FP32, what=f"int pulse {b}")


def test_single_lfm_pulse_d4_full(oracle):
    """One LFM pulse (TB = 64) at N = 1024, causal D4, J = 3, 10 dB: all 1024
    lags at scales 0..3 against the oracle; the peak at the injected delay."""
    w = inputs.single_lfm(N=1024, J=3, TB=64, snr_db=10.0, seed=1)
    r, lag, mag, norm = run_plan("d4", 1024, 3, w["refs"], w["y"], w["ref_ids"])
    _, _, no, ro, _ = oracle.correlate_batch(0, w["refs"][[0]].astype(np.complex128),
                                             w["y"].astype(np.complex128), 3, want_r=True)
    U.check_r(r[0], ro[0], what="lfm d4")
    D = int(w["delays"][0])
    assert lag[0, 0] == D
    for j in range(1, 4):
        assert min((lag[0, j] - D) % 1024, (D - lag[0, j]) % 1024) <= (1 << j)


@pytest.mark.parametrize("fname,fid", [("legall53", 1), ("cdf97", 2)])
def test_full_size_two_reference_batch_sampled(oracle, fname, fid):
    """4096 pulses x N = 8192, J = 5 (LFM TB = 256 and Barker-13 halves, 0-20 dB)
    in one launch; full r stored, a seeded sample of pulses checked."""
    w = inputs.two_ref_batch(B=4096, N=8192, J=5)
    r, lag, mag, norm = run_plan(fname, 8192, 5, w["refs"], w["y"], w["ref_ids"])
    sample = np.array([0, 5, 2047, 2048, 3001, 4095])
    X = w["refs"][w["ref_ids"][sample]].astype(np.complex128)
    Y = w["y"][sample].astype(np.complex128)
    lo, mo, no, ro, _ = oracle.correlate_batch(fid, X, Y, 5, want_r=True)
    for i, b in enumerate(sample):
        U.check_r(r[b], ro[i], what=f"{fname} pulse {b}")
        U.check_peak_lags(lag[b], ro[i], U.RTOL_FP32, what=f"{fname} pulse {b}")
        assert lag[b, 0] == w["delays"][b]


def test_peaks_without_r_equal_peaks_with_r():
    w = inputs.random_batch(n_refs=2, B=100, N=1024, J=4, seed=4)
    _, l1, m1, n1 = run_plan("cdf97", 1024, 4, w["refs"], w["y"], w["ref_ids"], want_r=False)
    _, l2, m2, n2 = run_plan("cdf97", 1024, 4, w["refs"], w["y"], w["ref_ids"], want_r=True)
    np.testing.assert_array_equal(l1, l2)
    np.testing.assert_array_equal(m1, m2)
    np.testing.assert_array_equal(n1, n2)


def test_deterministic_reruns_bitwise():
    w = inputs.random_batch(n_refs=3, B=200, N=512, J=3, seed=8)
    a = run_plan("legall53", 512, 3, w["refs"], w["y"], w["ref_ids"])
    b = run_plan("legall53", 512, 3, w["refs"], w["y"], w["ref_ids"])
    assert torch.equal(a[0].r, b[0].r)
    for u, v in zip(a[1:], b[1:]):
        np.testing.assert_array_equal(u, v)


def test_invalid_reference_id_is_isolated_and_reported():
    from paper_cs_0607001_gb300 import sidwt
    w = inputs.random_batch(n_refs=2, B=10, N=256, J=3, seed=3)
    ids = w["ref_ids"].copy()
    ids[4] = 7
    ids[6] = -1
    with sidwt.Plan("legall53", 256, 3) as p:
        for x in w["refs"]:
            p.store_reference(U.to_dev_c64(x))
        p.correlate(torch.from_numpy(ids).to(U.dev()), U.to_dev_c64(w["y"]))
        lag, mag, norm = p.peaks(10)
        torch.cuda.synchronize()
        lag = lag.cpu().numpy()
        assert (lag[4] == -1).all() and (lag[6] == -1).all()
        assert (lag[[0, 1, 2, 3, 5, 7, 8, 9]] >= 0).all()
        with pytest.raises(sidwt.SidwtError, match="EINVAL"):
            p.check()
        p.check()  # the record was cleared


def test_empty_batch_and_argument_errors():
    from paper_cs_0607001_gb300 import sidwt
    with sidwt.Plan("cdf97", 128, 3) as p:
        y = torch.zeros((0, 128), dtype=torch.complex64, device=U.dev())
        ids = torch.zeros(0, dtype=torch.int32, device=U.dev())
        with pytest.raises(sidwt.SidwtError, match="no stored reference"):
            p.correlate(torch.zeros(1, dtype=torch.int32, device=U.dev()),
                        torch.zeros((1, 128), dtype=torch.complex64, device=U.dev()))
        p.store_reference(torch.ones(128, dtype=torch.complex64, device=U.dev()))
        p.correlate(ids, y)
        lag, _, _ = p.peaks(0)
        assert lag.shape == (0, 4)
        with pytest.raises(sidwt.SidwtError, match="EINVAL"):
            p.peaks(3)
        with pytest.raises(sidwt.SidwtError, match="EINVAL"):
            p.correlate(torch.zeros(1, dtype=torch.int32, device=U.dev()),
                        torch.zeros((1, 128), dtype=torch.complex64, device=U.dev()), precision=7)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_host_entry_point_matches_device_entry_point(precision):
    w = inputs.random_batch(n_refs=2, B=64, N=1024, J=4, seed=12)
    from paper_cs_0607001_gb300 import sidwt
    with sidwt.Plan("legall53", 1024, 4) as p:
        for x in w["refs"]:
            p.store_reference(U.to_dev_c64(x))
        ids = torch.from_numpy(w["ref_ids"].astype(np.int32))
        y = torch.from_numpy(w["y"])
        lh, mh, nh = p.correlate_host(ids, y, precision=precision)  # pageable
        lp, mp, np_ = p.correlate_host(ids.pin_memory(), y.pin_memory(), precision=precision)  # pinned
        p.correlate(ids.to(U.dev()), y.to(U.dev()), precision=precision)
        ld, md, nd = p.peaks(64)
        torch.cuda.synchronize()
        for a, b in ((lh, ld), (mh, md), (nh, nd), (lp, ld)):
            np.testing.assert_array_equal(a.numpy(), b.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_async_host_entry_point_pipeline(precision):
    """Two plans on one stream, three rounds enqueued back to back with
    different pulses each round (the plan's device copy of the inputs is
    reused every round), one synchronisation at the end: every round's peaks
    equal the device entry point's on the same pulses."""
    from paper_cs_0607001_gb300 import sidwt
    N, J, B = 2048, 4, 96
    w3 = inputs.random_batch(n_refs=2, B=3 * B, N=N, J=J, seed=40)
    refs = w3["refs"]
    ws = [{key: w3[key][k * B:(k + 1) * B] for key in ("ref_ids", "y", "delays")} for k in range(3)]
    s = torch.cuda.Stream()
    with sidwt.Plan("legall53", N, J) as pa, sidwt.Plan("cdf97", N, J) as pb:
        for p in (pa, pb):
            for x in refs:
                p.store_reference(U.to_dev_c64(x))
        outs = []
        hin = [(torch.from_numpy(w["ref_ids"].astype(np.int32)).pin_memory(), torch.from_numpy(w["y"]).pin_memory())
               for w in ws]
        for k in range(3):
            for p in (pa, pb):
                o = tuple(torch.empty((B, J + 1), dtype=dt).pin_memory()
                          for dt in (torch.int32, torch.float32, torch.float64))
                p.correlate_host_async(hin[k][0], hin[k][1], *o, precision=precision, stream=s)
                outs.append((k, p, o))
        s.synchronize()
        with pytest.raises(ValueError, match="pinned"):
            pa.correlate_host_async(hin[0][0], torch.from_numpy(ws[0]["y"]), *outs[0][2], stream=s)
        for k, p, (lag, mag, norm) in outs:
            p.correlate(hin[k][0].to(U.dev()), hin[k][1].to(U.dev()), precision=precision)
            ld, md, nd = p.peaks(B)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(lag.numpy(), ld.cpu().numpy())
            np.testing.assert_array_equal(mag.numpy(), md.cpu().numpy())
            np.testing.assert_array_equal(norm.numpy(), nd.cpu().numpy())
            assert (lag.numpy()[:, 0] == ws[k]["delays"]).all()


def test_latency_path_repeated_calls_and_graph_replays():
    """Batches of at most 16 pulses: the latency kernel's last CTA forms the
    peak records and resets its finished-CTA count, so calls one after the
    other, and replays of a captured call, give the records of a fresh plan."""
    from paper_cs_0607001_gb300 import sidwt
    N, J, B = 512, 3, 5
    w = inputs.random_batch(n_refs=2, B=2 * B, N=N, J=J, seed=41)
    ids = [torch.from_numpy(w["ref_ids"][i * B:(i + 1) * B].copy()).to(U.dev()) for i in range(2)]
    ys = [U.to_dev_c64(w["y"][i * B:(i + 1) * B]) for i in range(2)]

    def fresh(i):
        with sidwt.Plan("cdf97", N, J) as q:
            for x in w["refs"]:
                q.store_reference(U.to_dev_c64(x))
            q.correlate(ids[i], ys[i])
            return [t.cpu().numpy() for t in q.peaks(B)]

    want = [fresh(0), fresh(1)]
    with sidwt.Plan("cdf97", N, J) as p:
        for x in w["refs"]:
            p.store_reference(U.to_dev_c64(x))
        for i in (0, 1, 0, 1):
            p.correlate(ids[i], ys[i])
            got = [t.cpu().numpy() for t in p.peaks(B)]
            for a, b in zip(got, want[i]):
                np.testing.assert_array_equal(a, b)
        lag = torch.empty((B, J + 1), dtype=torch.int32, device=U.dev())
        mag = torch.empty((B, J + 1), dtype=torch.float32, device=U.dev())
        norm = torch.empty((B, J + 1), dtype=torch.float64, device=U.dev())
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            p.correlate(ids[1], ys[1])
            p.peaks_into(B, lag, mag, norm)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            p.correlate(ids[1], ys[1])
            p.peaks_into(B, lag, mag, norm)
        for _ in range(3):
            lag.fill_(-7)
            g.replay()
            torch.cuda.synchronize()
            for a, b in zip((lag, mag, norm), want[1]):
                np.testing.assert_array_equal(a.cpu().numpy(), b)
        p.check()
