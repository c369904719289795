"""ctypes binding of the FP64 CPU oracle (``sidwt_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is the independent checker of the CUDA
library.  It is loaded by the tests, by ``__graft_entry__.smoke()`` and by the
CPU-baseline leg of ``bench.py``; the library itself never imports it.

Complex vectors cross this boundary as numpy ``complex128`` arrays (interleaved
re/im doubles).  Filter ids: 0 causal Daubechies-4 (eq. 17), 1 LeGall 5/3,
2 CDF 9/7 (Table I), 3 reversible integer LeGall 5/3, 4 integer CDF 9/7 (Table I's
steps as dyadic fractions, rounded updates).  Sides: 0 = stored signal
x (primal analysis), 1 = received signal y (dual analysis).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "sidwt_oracle.c"
BUILD_DIR = HERE / "_build"
LIB = BUILD_DIR / "libsidwt_oracle.so"

D4, LEGALL53, CDF97, LEGALL53_INT, CDF97_INT = 0, 1, 2, 3, 4
SIDE_X, SIDE_Y = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/_build."""
    BUILD_DIR.mkdir(exist_ok=True)
    if LIB.exists() and not force and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    tmp = LIB.with_suffix(f".so.{os.getpid()}")
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", str(tmp), str(SRC), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(LIB))
        L.oracle_lift_level.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_long, _dp, _dp]
        L.oracle_lift_level_inv.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_long, _dp]
        L.oracle_int53_level.argtypes = [ctypes.c_int, _i64p, ctypes.c_long, _i64p, _i64p]
        L.oracle_int53_level_inv.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_long, _i64p]
        L.oracle_mallat_level.argtypes = [_dp, ctypes.c_long, ctypes.c_int, _ip, _dp, ctypes.c_int, _ip, _dp,
                                          _dp, _dp]
        L.oracle_mallat_level.restype = None
        L.oracle_pyramid_y.argtypes = [ctypes.c_int, _dp, ctypes.c_long, ctypes.c_int, _dp, _dp]
        L.oracle_tree_x.argtypes = [ctypes.c_int, _dp, ctypes.c_long, ctypes.c_int, _dp, _dp]
        L.oracle_delayed_analysis_x.argtypes = [ctypes.c_int, _dp, ctypes.c_long, ctypes.c_int, ctypes.c_long,
                                                _dp, _dp]
        L.oracle_correlate.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_long, ctypes.c_int, _dp, ctypes.c_int]
        L.oracle_brute_xcorr.argtypes = [_dp, _dp, ctypes.c_long, _dp]
        L.oracle_brute_xcorr.restype = None
        L.oracle_correlate_batch.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_long, ctypes.c_long, ctypes.c_int,
                                             ctypes.c_int, _i32p, _dp, _dp, _dp, ctypes.c_int]
        _lp = ctypes.POINTER(ctypes.c_long)
        L.oracle_correlate_mixed.argtypes = [ctypes.c_long, _ip, _lp, _ip, _lp, _lp, _dp, _dp, _i32p, _dp, _dp,
                                             ctypes.c_int]
        L.oracle_cdf97_constants.argtypes = [_dp]
        L.oracle_cdf97_constants.restype = None
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _check(rc):
    if rc < 0:
        raise ValueError("oracle rejected the arguments")
    return rc


def set_cdf97_t(t: float) -> None:
    """Select the CDF 9/7 member with free parameter t (Sec. III-C Case II)
    for every later 9/7 call of this process; t = 0 restores Table I."""
    L = lib()
    L.oracle_set_cdf97_t.argtypes = [ctypes.c_double]
    _check(L.oracle_set_cdf97_t(float(t)))


def cdf97_constants() -> np.ndarray:
    out = np.zeros(5)
    lib().oracle_cdf97_constants(_d(out))
    return out


def lift_level(filter_id: int, side: int, v) -> tuple[np.ndarray, np.ndarray]:
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    K = v.shape[0]
    a = np.zeros(K // 2)
    b = np.zeros(K // 2)
    _check(lib().oracle_lift_level(filter_id, side, _d(v), K, _d(a), _d(b)))
    return a, b


def lift_level_inv(filter_id: int, side: int, a, b) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    v = np.zeros(2 * a.shape[0])
    _check(lib().oracle_lift_level_inv(filter_id, side, _d(a), _d(b), v.shape[0], _d(v)))
    return v


def int53_level(side: int, v) -> tuple[np.ndarray, np.ndarray]:
    v = np.ascontiguousarray(np.asarray(v, dtype=np.int64))
    K = v.shape[0]
    a = np.zeros(K // 2, np.int64)
    b = np.zeros(K // 2, np.int64)
    _check(lib().oracle_int53_level(side, v.ctypes.data_as(_i64p), K, a.ctypes.data_as(_i64p),
                                    b.ctypes.data_as(_i64p)))
    return a, b


def int97_level(side: int, v) -> tuple[np.ndarray, np.ndarray]:
    L = lib()
    L.oracle_int97_level.argtypes = [ctypes.c_int, _i64p, ctypes.c_long, _i64p, _i64p]
    v = np.ascontiguousarray(np.asarray(v, dtype=np.int64))
    a = np.zeros(v.shape[0] // 2, np.int64)
    b = np.zeros(v.shape[0] // 2, np.int64)
    _check(L.oracle_int97_level(side, v.ctypes.data_as(_i64p), v.shape[0], a.ctypes.data_as(_i64p),
                                b.ctypes.data_as(_i64p)))
    return a, b


def int97_level_inv(side: int, a, b) -> np.ndarray:
    L = lib()
    L.oracle_int97_level_inv.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_long, _i64p]
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.int64))
    v = np.zeros(2 * a.shape[0], np.int64)
    _check(L.oracle_int97_level_inv(side, a.ctypes.data_as(_i64p), b.ctypes.data_as(_i64p), v.shape[0],
                                    v.ctypes.data_as(_i64p)))
    return v


def int53_level_inv(side: int, a, b) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.int64))
    v = np.zeros(2 * a.shape[0], np.int64)
    _check(lib().oracle_int53_level_inv(side, a.ctypes.data_as(_i64p), b.ctypes.data_as(_i64p), v.shape[0],
                                        v.ctypes.data_as(_i64p)))
    return v


def mallat_level(v, lo: dict[int, float], hi: dict[int, float]) -> tuple[np.ndarray, np.ndarray]:
    """Convolution-and-downsample with caller-given taps {offset: value}."""
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    K = v.shape[0]
    ol = np.array(list(lo.keys()), dtype=np.intc)
    vl = np.array(list(lo.values()), dtype=np.float64)
    oh = np.array(list(hi.keys()), dtype=np.intc)
    vh = np.array(list(hi.values()), dtype=np.float64)
    a = np.zeros(K // 2)
    b = np.zeros(K // 2)
    lib().oracle_mallat_level(_d(v), K, len(ol), ol.ctypes.data_as(_ip), _d(vl), len(oh),
                              oh.ctypes.data_as(_ip), _d(vh), _d(a), _d(b))
    return a, b


def pyramid_y(filter_id: int, y, J: int) -> tuple[np.ndarray, np.ndarray]:
    """Received pyramid: level j at offset 2N - 4(N>>j): c_j then d_j (complex)."""
    y = _c128(y)
    N = y.shape[0]
    out = np.zeros(2 * N - 2 * (N >> J), np.complex128)
    en = np.zeros(J + 1)
    _check(lib().oracle_pyramid_y(filter_id, _d(y.view(np.float64)), N, J, _d(out.view(np.float64)), _d(en)))
    return out, en


def pyramid_level(pyr: np.ndarray, N: int, j: int) -> tuple[np.ndarray, np.ndarray]:
    K = N >> j
    off = 2 * N - 4 * K
    return pyr[off:off + K], pyr[off + K:off + 2 * K]


def tree_x(filter_id: int, x, J: int) -> tuple[np.ndarray, np.ndarray]:
    """SIDWT tree: level j (1..J) at offset 2N(j-1): A[2^j][N>>j] then B[2^j][N>>j]."""
    x = _c128(x)
    N = x.shape[0]
    out = np.zeros(2 * N * J, np.complex128)
    en = np.zeros((2 << J) - 1)
    _check(lib().oracle_tree_x(filter_id, _d(x.view(np.float64)), N, J, _d(out.view(np.float64)), _d(en)))
    return out, en


def tree_level(tree: np.ndarray, N: int, j: int) -> tuple[np.ndarray, np.ndarray]:
    """(A, B) of level j, each shaped [2^j, N>>j]."""
    base = 2 * N * (j - 1)
    A = tree[base:base + N].reshape(1 << j, N >> j)
    B = tree[base + N:base + 2 * N].reshape(1 << j, N >> j)
    return A, B


def delayed_analysis_x(filter_id: int, x, j: int, D: int) -> tuple[np.ndarray, np.ndarray | None]:
    x = _c128(x)
    N = x.shape[0]
    out = np.zeros(N >> j, np.complex128)
    det = np.zeros(N >> j, np.complex128) if j >= 1 else None
    _check(lib().oracle_delayed_analysis_x(filter_id, _d(x.view(np.float64)), N, j, D, _d(out.view(np.float64)),
                                           _d(det.view(np.float64)) if det is not None else None))
    return out, det


def correlate(filter_id: int, x, y, J: int, form: int = 1) -> np.ndarray:
    """r[j][D] for j = 0..J, D = 0..N-1 (form 0: level-j definition; 1: eq. 20/20a)."""
    x = _c128(x)
    y = _c128(y)
    N = x.shape[0]
    r = np.zeros((J + 1, N), np.complex128)
    _check(lib().oracle_correlate(filter_id, _d(x.view(np.float64)), _d(y.view(np.float64)), N, J,
                                  _d(r.view(np.float64)), form))
    return r


def brute_xcorr(x, y) -> np.ndarray:
    x = _c128(x)
    y = _c128(y)
    r = np.zeros(x.shape[0], np.complex128)
    lib().oracle_brute_xcorr(_d(x.view(np.float64)), _d(y.view(np.float64)), x.shape[0], _d(r.view(np.float64)))
    return r


def correlate_batch(filter_id: int, X, Y, J: int, form: int = 1, want_r: bool = False, nthreads: int = 0):
    """Peaks of P pairs: returns (lag[P,J+1], mag[P,J+1], norm[P,J+1], r or None, threads used)."""
    X = _c128(X)
    Y = _c128(Y)
    P, N = X.shape
    lag = np.zeros((P, J + 1), np.int32)
    mag = np.zeros((P, J + 1))
    norm = np.zeros((P, J + 1))
    r = np.zeros((P, J + 1, N), np.complex128) if want_r else None
    used = _check(lib().oracle_correlate_batch(
        filter_id, _d(X.view(np.float64)), _d(Y.view(np.float64)), P, N, J, form, lag.ctypes.data_as(_i32p),
        _d(mag), _d(norm), _d(r.view(np.float64)) if r is not None else None, nthreads))
    return lag, mag, norm, r, used


def correlate_mixed(filters, Ns, Js, x_packed, y_packed, offsets, nthreads: int = 0):
    """Peaks of pairs of mixed shapes (packed complex inputs): returns
    (lag, mag, norm) packed by slot (pair i's J_i + 1 scales) and threads used."""
    f = np.ascontiguousarray(np.asarray(filters, dtype=np.intc))
    n = np.ascontiguousarray(np.asarray(Ns, dtype=np.int_))
    j = np.ascontiguousarray(np.asarray(Js, dtype=np.intc))
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int_))
    slot = np.ascontiguousarray(np.concatenate([[0], np.cumsum(j + 1)[:-1]]).astype(np.int_))
    S = int((j + 1).sum())
    X = _c128(x_packed)
    Y = _c128(y_packed)
    lag = np.zeros(S, np.int32)
    mag = np.zeros(S)
    norm = np.zeros(S)
    lp = ctypes.POINTER(ctypes.c_long)
    used = _check(lib().oracle_correlate_mixed(
        len(f), f.ctypes.data_as(_ip), n.ctypes.data_as(lp), j.ctypes.data_as(_ip), off.ctypes.data_as(lp),
        slot.ctypes.data_as(lp), _d(X.view(np.float64)), _d(Y.view(np.float64)), lag.ctypes.data_as(_i32p), _d(mag),
        _d(norm), nthreads))
    return lag, mag, norm, used
