"""Pins of the oracle's SIDWT tree, received pyramid and correlation.

  * shift-circulant identity (Sec. II): the tree's variants equal the analysis
    of x literally delayed by every D;
  * eq. 4 at full depth: sum_j <B_j, d_j> + <A_J, c_J> = <x, y>;
  * scale 0 equals the textbook circular cross-correlation;
  * the level-j definition and the paper's eq. 20 / 20a form agree;
  * the peak lands on the injected delay (Sec. IV, scale-invariant peak);
  * the reversible integer path is exact and close to the float 5/3 path.
"""
import numpy as np
import pytest

from paper_cs_0607001_gb300 import inputs

FILTERS = [0, 1, 2, 3, 4]


def crand(g, n):
    return g.standard_normal(n) + 1j * g.standard_normal(n)


def signal_for(f, g, N):
    if f in (3, 4):
        return (g.integers(-2000, 2000, size=N) + 1j * g.integers(-2000, 2000, size=N)).astype(np.complex128)
    return crand(g, N)


@pytest.mark.parametrize("f", FILTERS)
@pytest.mark.parametrize("N,J", [(16, 2), (32, 3), (64, 4)])
def test_tree_variants_equal_brute_force_delays(oracle, f, N, J):
    g = np.random.default_rng(N + f)
    x = signal_for(f, g, N)
    tree, en = oracle.tree_x(f, x, J)
    for j in range(1, J + 1):
        A, B = oracle.tree_level(tree, N, j)
        for D in range(N):
            r, q = D % (1 << j), D // (1 << j)
            a, b = oracle.delayed_analysis_x(f, x, j, D)
            np.testing.assert_allclose(np.roll(A[r], q), a, rtol=0, atol=1e-11 * max(1, np.abs(x).max()))
            np.testing.assert_allclose(np.roll(B[r], q), b, rtol=0, atol=1e-11 * max(1, np.abs(x).max()))
        for r in range(1 << j):
            assert en[(1 << j) - 1 + r] == pytest.approx(np.vdot(A[r], A[r]).real, rel=1e-12)


@pytest.mark.parametrize("f", [0, 1, 2])
@pytest.mark.parametrize("N,J", [(8, 3), (64, 3), (256, 5), (1024, 10)])
def test_full_depth_parseval(oracle, f, N, J):
    """eq. 4: the DWT-domain inner product equals <x, y>."""
    g = np.random.default_rng(N * 3 + f)
    x, y = crand(g, N), crand(g, N)
    tree, _ = oracle.tree_x(f, x, J)
    pyr, _ = oracle.pyramid_y(f, y, J)
    s = 0j
    for j in range(1, J + 1):
        A, B = oracle.tree_level(tree, N, j)
        c, d = oracle.pyramid_level(pyr, N, j)
        s += np.vdot(B[0], d)
        if j == J:
            s += np.vdot(A[0], c)
    ref = np.vdot(x, y)
    assert abs(s - ref) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)


@pytest.mark.parametrize("f", FILTERS)
@pytest.mark.parametrize("N,J", [(16, 1), (32, 5), (128, 3), (96, 5), (2, 1), (128, 1)])
def test_correlation_forms_agree_and_scale0_is_brute_force(oracle, f, N, J):
    g = np.random.default_rng(7 * N + f)
    x = signal_for(f, g, N)
    y = signal_for(f, g, N)
    r0 = oracle.correlate(f, x, y, J, form=0)
    r1 = oracle.correlate(f, x, y, J, form=1)
    scale = np.linalg.norm(x) * np.linalg.norm(y)
    if f in (3, 4):
        # integer bands: the level-(j+1) form pairs integer details whose
        # scalings cancel, but the floor rounding makes the two forms differ
        # by a rounding-sized amount.  Each rounded step moves a coefficient
        # by less than one unit (at most four steps a level), so the forms
        # differ by about 4 J sqrt(N) (|x| + |y|) at most; for all but the
        # shortest signals that is well under 1e-3 |x| |y|
        tol = 1e-3 * scale if N >= 16 else 4 * J * np.sqrt(N) * (np.linalg.norm(x) + np.linalg.norm(y))
        assert np.abs(r0 - r1).max() <= tol
    else:
        assert np.abs(r0 - r1).max() <= 1e-12 * scale
    br = oracle.brute_xcorr(x, y)
    assert np.abs(r0[0] - br).max() <= 1e-12 * scale


@pytest.mark.parametrize("f", [0, 1, 2])
def test_scale_j_definition_by_hand(oracle, f):
    """r_j[D] = <level-j analysis of x delayed by D, level-j approximation of y>,
    computed here by literally delaying x for a few (j, D)."""
    N, J = 64, 4
    g = np.random.default_rng(11 + f)
    x, y = crand(g, N), crand(g, N)
    r = oracle.correlate(f, x, y, J, form=1)
    pyr, _ = oracle.pyramid_y(f, y, J)
    for j in range(1, J + 1):
        cj, _ = oracle.pyramid_level(pyr, N, j)
        for D in (0, 1, 5, 17, 63):
            a, _ = oracle.delayed_analysis_x(f, x, j, D)
            assert abs(np.vdot(a, cj) - r[j, D]) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)


def test_complex_is_real_transform_on_re_and_im(oracle):
    """Sec. IV / eq. 19: the complex DWT is the real DWT of Re plus i times that of Im."""
    g = np.random.default_rng(3)
    y = crand(g, 128)
    for f in (0, 1, 2):
        p, _ = oracle.pyramid_y(f, y, 4)
        pr, _ = oracle.pyramid_y(f, y.real.astype(np.complex128), 4)
        pi, _ = oracle.pyramid_y(f, y.imag.astype(np.complex128), 4)
        np.testing.assert_allclose(p, pr + 1j * pi, atol=1e-13)


@pytest.mark.parametrize("f", [0, 1, 2])
def test_peak_at_injected_delay(oracle, f):
    """Scale 0: the peak lag equals the injected delay exactly.  Coarser
    scales: within 2^j samples circularly (the shift-variance of the
    critically sampled tree is removed by the SIDWT only up to the scale's
    own resolution)."""
    N, J = 1024, 3
    for seed in range(3):
        w = inputs.single_lfm(N=N, J=J, TB=64, snr_db=10.0, seed=100 + seed)
        x = w["refs"][0].astype(np.complex128)
        y = w["y"][0].astype(np.complex128)
        D = int(w["delays"][0])
        lag, mag, norm, _, _ = oracle.correlate_batch(f, x[None], y[None], J)
        assert lag[0, 0] == D
        for j in range(1, J + 1):
            dist = min((lag[0, j] - D) % N, (D - lag[0, j]) % N)
            assert dist <= (1 << j), (f, j, lag[0], D)
        assert np.all(norm[0] <= 1.0 + 1e-12)
        assert norm[0, 0] > 0.5


def test_noiseless_echo_normalised_peak_is_one(oracle):
    N, J = 256, 4
    x = inputs.lfm(N, 64)
    y = np.roll(x, 77)
    for f in (0, 1, 2):
        lag, mag, norm, _, _ = oracle.correlate_batch(f, x[None], y[None], J)
        assert lag[0, 0] == 77
        assert norm[0, 0] == pytest.approx(1.0, abs=1e-12)
        # orthogonal D4 uses the same transform on both sides, so the level-j
        # bands of the echo equal the stored variant's and Cauchy-Schwarz is
        # tight at every scale; the biorthogonal pairs are tight at scale 0 only
        for j in range(J + 1):
            if f == 0 and lag[0, j] == 77:
                assert norm[0, j] == pytest.approx(1.0, abs=1e-12)
            assert norm[0, j] <= 1.0 + 1e-12


@pytest.mark.parametrize("N,J", [(64, 3), (1024, 5)])
def test_int53_pyramid_reversible_and_exact(oracle, N, J):
    g = np.random.default_rng(N)
    y = (g.integers(-32768, 32768, size=N) + 1j * g.integers(-32768, 32768, size=N)).astype(np.complex128)
    pyr, _ = oracle.pyramid_y(3, y, J)
    assert np.all(pyr.real == np.round(pyr.real)) and np.all(pyr.imag == np.round(pyr.imag))
    # reconstruct level by level with the integer inverse
    c, _ = oracle.pyramid_level(pyr, N, J)
    cur = c
    for j in range(J, 0, -1):
        _, d = oracle.pyramid_level(pyr, N, j)
        re = oracle.int53_level_inv(1, cur.real.astype(np.int64), d.real.astype(np.int64))
        im = oracle.int53_level_inv(1, cur.imag.astype(np.int64), d.imag.astype(np.int64))
        cur = re + 1j * im
    np.testing.assert_array_equal(cur, y)


def test_int_path_correlation_close_to_float(oracle):
    N, J = 512, 4
    w = inputs.single_lfm(N=N, J=J, TB=128, snr_db=15.0, seed=5)
    xi = inputs.to_iq16(w["refs"][0])[0]
    yi = inputs.to_iq16(w["y"][0])[0]
    x = xi[:, 0] + 1j * xi[:, 1].astype(np.float64)
    y = yi[:, 0] + 1j * yi[:, 1].astype(np.float64)
    ri = oracle.correlate(3, x, y, J, form=1)
    rf = oracle.correlate(1, x, y, J, form=1)
    # floor rounding adds about half a unit per coefficient and per level, so
    # the deviation from the exact float 5/3 grows roughly like 2^j
    for j in range(J + 1):
        assert np.abs(ri[j] - rf[j]).max() <= 1e-5 * 2 ** (j + 1) * np.abs(rf[j]).max()
    assert int(np.argmax(np.abs(ri[0]))) == int(w["delays"][0])


def test_batch_matches_single_and_uses_threads(oracle):
    g = np.random.default_rng(2)
    X = np.stack([crand(g, 64) for _ in range(5)])
    Y = np.stack([np.roll(X[i], 7 * i + 1) + 0.1 * crand(g, 64) for i in range(5)])
    lag, mag, norm, r, used = oracle.correlate_batch(2, X, Y, 3, want_r=True)
    assert used >= 1
    for i in range(5):
        ri = oracle.correlate(2, X[i], Y[i], 3)
        np.testing.assert_allclose(r[i], ri, atol=1e-12)
        assert lag[i, 0] == 7 * i + 1
        for j in range(4):
            m = np.abs(ri[j])
            assert mag[i, j] == pytest.approx(m.max())
            assert lag[i, j] == int(np.argmax(m))


def test_bad_shapes_rejected(oracle):
    with pytest.raises(ValueError):
        oracle.correlate(1, np.zeros(12), np.zeros(12), 3)
    with pytest.raises(ValueError):
        oracle.pyramid_y(7, np.zeros(16), 2)
