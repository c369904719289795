"""GPU parity of the ragged path's full correlation output
(sidwt_ragged_correlate_r): r_j[D] at every lag D and every scale j of every
pulse, element by element against the FP64 oracle.

The batch has 22 pulses of mixed filter, length and depth: bands that are a
multiple of 64 (the tensor-core kernel's circular form), bands of 64 or more
that are not (its zero-padded linear form), bands under 64 (the CUDA-core
kernel), and scale pairs J - 1 / J at the same tile width (scale J formed
from band 0 of scale J - 1's tiles).  Each tensor-core tile width S in
{256, 192, 128, 64} is forced in turn through the tuning cache.  BF16x3 is held
to the split's worst-case and per-MMA-step bounds (tests/gpu_util.py), FP32
to 1e-5 of each (pulse, scale)'s largest |r|.  The peak records of the same
call are checked against the call's own r: the reported lag is a maximum of
|r_gpu| and the reported magnitude is |r_gpu| there.
"""
import numpy as np
import pytest
import torch

from tests import gpu_util as U

# (filter id, N, J)
SPECS = [(1, 2048, 3), (2, 8000, 3), (0, 4096, 4), (1, 3000, 2), (2, 1536, 5), (0, 512, 3), (2, 96, 5),
         (1, 6144, 3), (0, 1024, 1), (2, 3000, 2), (1, 640, 2), (2, 704, 6), (0, 12288, 5), (1, 2560, 4),
         (2, 4000, 5), (0, 7168, 3), (1, 192, 1), (2, 16384, 6), (0, 2304, 2), (1, 5120, 5), (2, 1152, 3),
         (0, 10000, 4)]


def band_kinds():
    """Which paths the batch covers: (circular, zero-padded, CUDA-core) band counts."""
    circ = pad = simt = 0
    for _, N, J in SPECS:
        for j in range(J + 1):
            Kp = N >> (j + 1 if j < J else J)
            if Kp < 64:
                simt += 1
            elif Kp % 64 == 0:
                circ += 1
            else:
                pad += 1
    return circ, pad, simt


def test_batch_covers_every_band_kind():
    circ, pad, simt = band_kinds()
    assert len(SPECS) >= 20 and circ >= 20 and pad >= 10 and simt >= 5


@pytest.fixture(scope="module")
def batch(oracle):
    g = np.random.default_rng(77)
    refs, ys, delays = [], [], []
    for f, N, J in SPECS:
        x = ((g.standard_normal(N) + 1j * g.standard_normal(N)) / np.sqrt(2)).astype(np.complex64)
        D = int(g.integers(0, N))
        y = (np.roll(x, D) + 0.4 * (g.standard_normal(N) + 1j * g.standard_normal(N))).astype(np.complex64)
        refs.append(x)
        ys.append(y)
        delays.append(D)
    offsets = np.concatenate([[0], np.cumsum([s[1] for s in SPECS])[:-1]]).astype(np.int64)
    ref_r, bounds = [], []
    for (f, N, J), x, y in zip(SPECS, refs, ys):
        x64, y64 = x.astype(np.complex128), y.astype(np.complex128)
        ref_r.append(oracle.correlate(f, x64, y64, J))
        tree, _ = oracle.tree_x(f, x64, J)
        pyr, _ = oracle.pyramid_y(f, y64, J)
        bounds.append([U.split_bounds(tree, pyr, N, J, j, 2.0 ** -16) for j in range(J + 1)])
    return refs, np.concatenate(ys), offsets, delays, ref_r, bounds


def run_r(precision, refs, ypack, offsets, split="auto"):
    from paper_cs_0607001_gb300 import sidwt
    with sidwt.Ragged() as rg:
        rg.set_precision(precision)
        rg.set_split(split)
        ids = [rg.store_reference(f, N, J, U.to_dev_c64(x)) for (f, N, J), x in zip(SPECS, refs)]
        n, r = rg.correlate_r(ids, offsets, U.to_dev_c64(ypack))
        lag, mag, _ = rg.peaks(n)
        rg.check()
        first_slot, _ = rg.slots_of(ids)
        first_r, total = rg.r_rows_of(ids)
        torch.cuda.synchronize()
        return (first_slot, first_r, r.cpu().numpy().astype(np.complex128), lag.cpu().numpy(), mag.cpu().numpy())


def check(precision, batch, split="auto"):
    refs, ypack, offsets, delays, ref_r, bounds = batch
    first_slot, first_r, r, lag, mag = run_r(precision, refs, ypack, offsets, split)
    worst_ratio = 0.0
    for i, (f, N, J) in enumerate(SPECS):
        for j in range(J + 1):
            got = r[first_r[i] + j * N:first_r[i] + (j + 1) * N]
            want = ref_r[i][j]
            err = np.abs(got - want).max()
            top = np.abs(want).max()
            what = f"item {i} {SPECS[i]} scale {j}"
            if precision == "fp32":
                assert err <= U.RTOL_FP32 * top, f"{what}: {err:.3e} > 1e-5 x {top:.3e}"
            else:
                worst, step = bounds[i][j]
                assert err <= worst, f"{what}: {err:.3e} > worst-case bound {worst:.3e}"
                assert err <= step, f"{what}: {err:.3e} > per-MMA-step bound {step:.3e}"
                worst_ratio = max(worst_ratio, err / step)
            # the call's peak record against its own r
            s = first_slot[i] + j
            a = np.abs(got)
            # (rows of the tensor-core tiles that repeat an advance sum it in another order)
            assert 0 <= lag[s] < N and a[lag[s]] >= a.max() * (1 - 1e-5), what
            assert mag[s] == pytest.approx(a[lag[s]], rel=1e-5, abs=1e-30), what
        assert lag[first_slot[i]] == delays[i], f"item {i}: scale-0 peak off the injected delay"
    return worst_ratio


@pytest.mark.gpu
@pytest.mark.parametrize("width", [256, 192, 128, 64])
def test_ragged_bf16x3_full_r_each_tile_width(batch, tmp_path, monkeypatch, width):
    lines = [f"tc {S} {lg} {1.0 if S == width else 50.0}" for S in (256, 192, 128, 64) for lg in range(25)]
    cache = tmp_path / "forced.txt"
    cache.write_text("\n".join(lines) + "\n")
    monkeypatch.setenv("SIDWT_TUNE_CACHE", str(cache))
    check("bf16x3", batch)


@pytest.mark.gpu
def test_ragged_bf16x3_full_r_default_widths(batch):
    check("bf16x3", batch)


@pytest.mark.gpu
@pytest.mark.parametrize("split", ["always", "never"])
def test_ragged_bf16x3_full_r_split_contractions(batch, split):
    """Every tensor-core tile long enough cut into parts of its contraction
    (each part's accumulators summed by the reduction kernel, band-0 parts
    alone for the folded scale J), and no tile cut: the same bounds, peaks
    consistent with the call's own r.  (This 22-pulse batch has fewer tiles
    than SMs, so the default already splits.)"""
    check("bf16x3", batch, split)


@pytest.mark.gpu
def test_ragged_fp32_full_r(batch):
    check("fp32", batch)


@pytest.mark.gpu
def test_ragged_r_output_too_small_is_rejected():
    from paper_cs_0607001_gb300 import sidwt
    L = sidwt.lib()
    with sidwt.Ragged() as rg:
        x = torch.zeros(256, dtype=torch.complex64, device=U.dev())
        rid = rg.store_reference("cdf97", 256, 3, x)
        ids = np.array([rid], np.int32)
        off = np.zeros(1, np.int64)
        r = torch.zeros(4 * 256 - 1, dtype=torch.complex64, device=U.dev())
        st = L.sidwt_ragged_correlate_r(rg._h, 1, ids.ctypes.data, off.ctypes.data, x.data_ptr(), 256,
                                        r.data_ptr(), r.numel(), torch.cuda.current_stream().cuda_stream)
        assert st == 1 and b"r_dev holds" in L.sidwt_last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_batched_store_equals_one_by_one_store(batch, precision):
    """sidwt_ragged_store_references (all trees of a batch built together)
    gives the same stored trees, energies and packed operands as storing the
    signals one at a time: the same batch's peaks are bit-identical, and so is
    r up to which of the tensor-core tiles' repeated advances (each summed in
    its own order) lands last."""
    from paper_cs_0607001_gb300 import sidwt
    refs, ypack, offsets, delays, ref_r, bounds = batch
    xpack = U.to_dev_c64(np.concatenate(refs))
    yd = U.to_dev_c64(ypack)
    out = []
    for batched in (False, True):
        with sidwt.Ragged() as rg:
            rg.set_precision(precision)
            if batched:
                ids = rg.store_references([s[0] for s in SPECS], [s[1] for s in SPECS], [s[2] for s in SPECS], xpack,
                                          offsets)
            else:
                ids = [rg.store_reference(f, N, J, xpack[o:o + N]) for (f, N, J), o in zip(SPECS, offsets)]
            n, r = rg.correlate_r(ids, offsets, yd)
            lag, mag, norm = rg.peaks(n)
            rg.check()
            torch.cuda.synchronize()
            out.append((r.cpu().numpy(), lag.cpu().numpy(), mag.cpu().numpy(), norm.cpu().numpy()))
    for a, b in zip(out[0][1:], out[1][1:]):
        np.testing.assert_array_equal(a, b)
    r0, r1 = out[0][0], out[1][0]
    if precision == "fp32":
        np.testing.assert_array_equal(r0, r1)
    else:
        assert np.abs(r0 - r1).max() <= 1e-6 * np.abs(r0).max()
