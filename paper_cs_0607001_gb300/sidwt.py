"""Thin ctypes binding of libsidwt (include/sidwt.h).

Argument marshalling only: every step of the correlation runs in the CUDA
library.  PyTorch supplies device memory and the current CUDA stream.  The
binding raises if the compiled library is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np
import torch

from . import build as _build

FILTERS = {"d4": 0, "legall53": 1, "cdf97": 2, "legall53_int": 3, "cdf97_int": 4}
PRECISIONS = {"fp32": 0, "bf16x3": 1, "tf32x3": 2}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EBUSY", 6: "EUNSUPPORTED"}


class SidwtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Timing(ctypes.Structure):
    _fields_ = [("store_ms", ctypes.c_double), ("group_ms", ctypes.c_double), ("analyze_ms", ctypes.c_double),
                ("correlate_ms", ctypes.c_double), ("peaks_ms", ctypes.c_double),
                ("correlate_calls", ctypes.c_int64), ("launches", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("max_j", ctypes.c_int32),
                ("memory_cap_bytes", ctypes.c_int64), ("max_lane_samples", ctypes.c_int64),
                ("precision", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("rejected", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("max_batch", ctypes.c_int64), ("samples", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("span_s", ctypes.c_double), ("ref_hits", ctypes.c_int64), ("ref_stores", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


def library_path() -> Path:
    return _build.LIB


def lib():
    """Load libsidwt.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not path.exists():
        raise RuntimeError(f"libsidwt is not built ({path} missing): run __graft_entry__.build() first")
    L = ctypes.CDLL(str(path))
    L.sidwt_version.restype = ctypes.c_char_p
    L.sidwt_last_error.restype = ctypes.c_char_p
    L.sidwt_plan_create.argtypes = [ctypes.c_int, _i64, ctypes.c_int, ctypes.POINTER(_vp)]
    L.sidwt_plan_destroy.argtypes = [_vp]
    L.sidwt_plan_reserve.argtypes = [_vp, _i32, _i64]
    L.sidwt_plan_num_refs.argtypes = [_vp]
    L.sidwt_plan_num_refs.restype = _i32
    L.sidwt_store_reference.argtypes = [_vp, _vp, ctypes.POINTER(_i32), _vp]
    L.sidwt_reference_tree.argtypes = [_vp, _i32, _vp, _vp, _vp]
    L.sidwt_analyze.argtypes = [_vp, _vp, _i64, _vp, _vp, _vp]
    L.sidwt_correlate.argtypes = [_vp, _vp, _vp, _i64, ctypes.c_int, _vp, _vp]
    L.sidwt_correlate_again.argtypes = [_vp, _vp, _i64, ctypes.c_int, _vp, _vp]
    L.sidwt_peaks.argtypes = [_vp, _i64, _vp, _vp, _vp, _vp]
    L.sidwt_correlate_host.argtypes = [_vp, _vp, _vp, _i64, ctypes.c_int, _vp, _vp, _vp, _vp]
    L.sidwt_correlate_host_async.argtypes = [_vp, _vp, _vp, _i64, ctypes.c_int, _vp, _vp, _vp, _vp]
    L.sidwt_check.argtypes = [_vp, _vp]
    L.sidwt_reset_references.argtypes = [_vp]
    L.sidwt_set_timing.argtypes = [_vp, ctypes.c_int]
    L.sidwt_read_timing.argtypes = [_vp, ctypes.POINTER(Timing), ctypes.c_int]
    L.sidwt_correlate_static.argtypes = [ctypes.c_int, _i64, ctypes.c_int, _vp, _vp, _i64, _vp, _vp, _vp, _vp]
    L.sidwt_tc_selftest.argtypes = [_vp, _vp, _vp]
    L.sidwt_debug_stall.argtypes = [ctypes.c_uint32]
    L.sidwt_synthesize.argtypes = [ctypes.c_int, _i64, _i64, _vp, _vp, _i64, _vp, _vp]
    L.sidwt_correlate_c2f.argtypes = [_vp, _vp, _vp, _i64, ctypes.c_int, _vp, _vp, _vp]
    L.sidwt_plan_set_cdf97_t.argtypes = [_vp, ctypes.c_double]
    L.sidwt_detect.argtypes = [_vp, _i64, _i64, ctypes.c_float, ctypes.c_int, _vp, _vp, _vp, _vp]
    L.sidwt_ragged_create.argtypes = [ctypes.POINTER(_vp)]
    L.sidwt_ragged_destroy.argtypes = [_vp]
    L.sidwt_ragged_reserve.argtypes = [_vp, _i64, _i64, _i64]
    L.sidwt_ragged_num_refs.argtypes = [_vp]
    L.sidwt_ragged_num_refs.restype = _i32
    L.sidwt_ragged_store_reference.argtypes = [_vp, ctypes.c_int, _i64, ctypes.c_int, _vp, ctypes.POINTER(_i32), _vp]
    L.sidwt_ragged_store_references.argtypes = [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp]
    L.sidwt_ragged_correlate.argtypes = [_vp, _i64, _vp, _vp, _vp, _i64, _vp]
    L.sidwt_ragged_correlate_r.argtypes = [_vp, _i64, _vp, _vp, _vp, _i64, _vp, _i64, _vp]
    L.sidwt_ragged_set_split.argtypes = [_vp, ctypes.c_int]
    L.sidwt_ragged_graph_create.argtypes = [_vp, _i64, _vp, _vp, _vp, _i64, ctypes.POINTER(_i32)]
    L.sidwt_ragged_graph_launch.argtypes = [_vp, _vp]
    L.sidwt_ragged_peaks.argtypes = [_vp, _i64, _vp, _vp, _vp, _vp]
    L.sidwt_ragged_autotune.argtypes = [_vp, ctypes.c_char_p, _vp]
    L.sidwt_ragged_tuning.argtypes = [_vp, _vp]
    L.sidwt_ragged_tc_weights.argtypes = [_vp, _vp]
    L.sidwt_ragged_set_timing.argtypes = [_vp, ctypes.c_int]
    L.sidwt_ragged_read_timing.argtypes = [_vp, ctypes.POINTER(Timing), ctypes.c_int]
    L.sidwt_ragged_reset_references.argtypes = [_vp]
    L.sidwt_ragged_set_precision.argtypes = [_vp, ctypes.c_int]
    L.sidwt_ragged_check.argtypes = [_vp, _vp]
    L.sidwt_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(_vp)]
    L.sidwt_server_add_waveform.argtypes = [_vp, _vp, _i64, ctypes.POINTER(_i32)]
    L.sidwt_server_start.argtypes = [_vp]
    L.sidwt_server_submit.argtypes = [_vp, _i32, ctypes.c_int, _i64, ctypes.c_int, _vp, ctypes.POINTER(_i64)]
    L.sidwt_server_wait.argtypes = [_vp, _i64, ctypes.c_double]
    L.sidwt_server_drain.argtypes = [_vp, ctypes.c_double]
    L.sidwt_server_result.argtypes = [_vp, _i64, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_double)]
    L.sidwt_server_forget.argtypes = [_vp, _i64]
    L.sidwt_server_read_stats.argtypes = [_vp, ctypes.POINTER(ServerStats), ctypes.c_int]
    L.sidwt_server_destroy.argtypes = [_vp]
    for name in ("sidwt_plan_create", "sidwt_plan_destroy", "sidwt_plan_reserve", "sidwt_store_reference",
                 "sidwt_reference_tree", "sidwt_analyze", "sidwt_correlate", "sidwt_correlate_again", "sidwt_peaks",
                 "sidwt_correlate_host", "sidwt_correlate_host_async", "sidwt_check", "sidwt_reset_references", "sidwt_set_timing",
                 "sidwt_read_timing", "sidwt_correlate_static", "sidwt_tc_selftest", "sidwt_debug_stall", "sidwt_ragged_create",
                 "sidwt_ragged_destroy", "sidwt_ragged_reserve", "sidwt_ragged_store_reference",
                 "sidwt_ragged_store_references",
                 "sidwt_ragged_correlate", "sidwt_ragged_correlate_r", "sidwt_ragged_set_split", "sidwt_ragged_graph_create", "sidwt_ragged_graph_launch",
                 "sidwt_ragged_peaks", "sidwt_ragged_autotune", "sidwt_ragged_tuning", "sidwt_ragged_set_timing",
                 "sidwt_ragged_read_timing", "sidwt_ragged_reset_references", "sidwt_server_create",
                 "sidwt_server_add_waveform", "sidwt_server_start", "sidwt_server_submit", "sidwt_server_wait",
                 "sidwt_server_drain", "sidwt_server_result", "sidwt_server_forget", "sidwt_server_read_stats",
                 "sidwt_server_destroy"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def version() -> str:
    return lib().sidwt_version().decode()


def _raise(status: int):
    if status != 0:
        raise SidwtError(status, lib().sidwt_last_error().decode())


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _filter_id(f) -> int:
    return FILTERS[f] if isinstance(f, str) else int(f)


def _prec_id(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


class Plan:
    """A correlation plan: filter, pulse length N, depth J, and the resident
    reference store (Sec. II-IV).  Device tensors must live on the current
    CUDA device; complex pulses are complex64, integer pulses int16 [.., N, 2]."""

    def __init__(self, filter, N: int, J: int):
        self.filter = _filter_id(filter)
        self.N = int(N)
        self.J = int(J)
        self.is_int = self.filter in (3, 4)
        h = _vp()
        _raise(lib().sidwt_plan_create(self.filter, self.N, self.J, ctypes.byref(h)))
        self._h = h

    # -- lifetime -----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().sidwt_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    @property
    def num_refs(self) -> int:
        return lib().sidwt_plan_num_refs(self._h)

    @property
    def pyr_elems(self) -> int:
        return 2 * self.N - 2 * (self.N >> self.J)

    def reserve(self, max_refs: int, max_batch: int):
        _raise(lib().sidwt_plan_reserve(self._h, max_refs, max_batch))

    # -- reference store ----------------------------------------------------
    def _check_pulses(self, t: torch.Tensor, batched: bool):
        if not t.is_cuda:
            raise ValueError("pulses must be CUDA tensors")
        if self.is_int:
            if t.dtype != torch.int16 or t.shape[-2:] != (self.N, 2):
                raise ValueError(f"integer plan expects int16 [..., {self.N}, 2]")
        else:
            if t.dtype != torch.complex64 or t.shape[-1] != self.N:
                raise ValueError(f"float plan expects complex64 [..., {self.N}]")
        if not t.is_contiguous():
            raise ValueError("pulses must be contiguous")

    def store_reference(self, x: torch.Tensor, stream=None) -> int:
        self._check_pulses(x, False)
        rid = _i32(-1)
        _raise(lib().sidwt_store_reference(self._h, _ptr(x), ctypes.byref(rid), _stream(stream)))
        return rid.value

    def reference_tree(self, ref_id: int, stream=None):
        dev = torch.cuda.current_device()
        n = 2 * self.J * self.N
        if self.is_int:
            tree = torch.empty((n, 2), dtype=torch.int32, device=dev)
        else:
            tree = torch.empty(n, dtype=torch.complex64, device=dev)
        en = torch.empty((2 << self.J) - 1, dtype=torch.float64, device=dev)
        _raise(lib().sidwt_reference_tree(self._h, ref_id, _ptr(tree), _ptr(en), _stream(stream)))
        return tree, en

    # -- received side --------------------------------------------------------
    def analyze(self, y: torch.Tensor, want_pyramid: bool = True, stream=None):
        self._check_pulses(y, True)
        B = y.shape[0]
        dev = y.device
        pyr = None
        if want_pyramid:
            if self.is_int:
                pyr = torch.empty((B, self.pyr_elems, 2), dtype=torch.int32, device=dev)
            else:
                pyr = torch.empty((B, self.pyr_elems), dtype=torch.complex64, device=dev)
        en = torch.empty((B, self.J + 1), dtype=torch.float64, device=dev)
        _raise(lib().sidwt_analyze(self._h, _ptr(y), B, _ptr(pyr), _ptr(en), _stream(stream)))
        return pyr, en

    def analyze_into(self, y: torch.Tensor, pyr=None, energies=None, stream=None):
        """Analysis into caller buffers (either may be None: kept in the plan only)."""
        _raise(lib().sidwt_analyze(self._h, _ptr(y), y.shape[0], _ptr(pyr), _ptr(energies), _stream(stream)))

    def correlate(self, ref_ids: torch.Tensor, y: torch.Tensor, precision="fp32", want_r: bool = False,
                  r_out: torch.Tensor | None = None, stream=None):
        self._check_pulses(y, True)
        B = y.shape[0]
        if ref_ids.dtype != torch.int32 or not ref_ids.is_cuda or ref_ids.numel() != B:
            raise ValueError("ref_ids must be a CUDA int32 tensor with one id per pulse")
        r = r_out
        if want_r and r is None:
            r = torch.empty((B, self.J + 1, self.N), dtype=torch.complex64, device=y.device)
        _raise(lib().sidwt_correlate(self._h, _ptr(ref_ids), _ptr(y), B, _prec_id(precision), _ptr(r),
                                     _stream(stream)))
        return r

    def correlate_again(self, ref_ids: torch.Tensor, precision="fp32", want_r: bool = False,
                        r_out: torch.Tensor | None = None, stream=None):
        """The pulses of the plan's last analysis against other stored signals
        (sidwt_correlate_again): no analysis is run."""
        B = ref_ids.numel()
        if ref_ids.dtype != torch.int32 or not ref_ids.is_cuda:
            raise ValueError("ref_ids must be a CUDA int32 tensor with one id per pulse")
        r = r_out
        if want_r and r is None:
            r = torch.empty((B, self.J + 1, self.N), dtype=torch.complex64, device=ref_ids.device)
        _raise(lib().sidwt_correlate_again(self._h, _ptr(ref_ids), B, _prec_id(precision), _ptr(r),
                                           _stream(stream)))
        return r

    def peaks(self, B: int, stream=None):
        dev = torch.cuda.current_device()
        lag = torch.empty((B, self.J + 1), dtype=torch.int32, device=dev)
        mag = torch.empty((B, self.J + 1), dtype=torch.float32, device=dev)
        norm = torch.empty((B, self.J + 1), dtype=torch.float64, device=dev)
        _raise(lib().sidwt_peaks(self._h, B, _ptr(lag), _ptr(mag), _ptr(norm), _stream(stream)))
        return lag, mag, norm

    def peaks_into(self, B: int, lag, mag, norm, stream=None):
        _raise(lib().sidwt_peaks(self._h, B, _ptr(lag), _ptr(mag), _ptr(norm), _stream(stream)))

    def correlate_host(self, ref_ids: torch.Tensor, y: torch.Tensor, precision="fp32", lag=None, mag=None,
                       norm=None, stream=None):
        """End-to-end call on host tensors (pinned or pageable): returns host peaks."""
        B = y.shape[0]
        if y.is_cuda or ref_ids.is_cuda:
            raise ValueError("correlate_host takes host tensors")
        if lag is None:
            lag = torch.empty((B, self.J + 1), dtype=torch.int32)
            mag = torch.empty((B, self.J + 1), dtype=torch.float32)
            norm = torch.empty((B, self.J + 1), dtype=torch.float64)
        _raise(lib().sidwt_correlate_host(self._h, _ptr(ref_ids), _ptr(y), B, _prec_id(precision), _ptr(lag),
                                          _ptr(mag), _ptr(norm), _stream(stream)))
        return lag, mag, norm

    def correlate_host_async(self, ref_ids: torch.Tensor, y: torch.Tensor, lag: torch.Tensor, mag: torch.Tensor,
                             norm: torch.Tensor, precision="fp32", stream=None):
        """Asynchronous end-to-end call on pinned host tensors
        (sidwt_correlate_host_async): the peaks land in lag / mag / norm once
        `stream` has been synchronised."""
        B = y.shape[0]
        for t in (ref_ids, y, lag, mag, norm):
            if t.is_cuda or not t.is_pinned():
                raise ValueError("correlate_host_async takes pinned host tensors")
        _raise(lib().sidwt_correlate_host_async(self._h, _ptr(ref_ids), _ptr(y), B, _prec_id(precision), _ptr(lag),
                                                _ptr(mag), _ptr(norm), _stream(stream)))

    def check(self, stream=None):
        _raise(lib().sidwt_check(self._h, _stream(stream)))

    def set_cdf97_t(self, t: float):
        """CDF 9/7 family member with free parameter t (0: Table I); before storing references."""
        _raise(lib().sidwt_plan_set_cdf97_t(self._h, float(t)))

    def correlate_c2f(self, ref_ids: torch.Tensor, y: torch.Tensor, half_window: int = 2, stream=None):
        """Coarse-to-fine peaks (sidwt_correlate_c2f): (lag, mag) [B][J+1]."""
        self._check_pulses(y, True)
        B = y.shape[0]
        lag = torch.empty((B, self.J + 1), dtype=torch.int32, device=y.device)
        mag = torch.empty((B, self.J + 1), dtype=torch.float32, device=y.device)
        _raise(lib().sidwt_correlate_c2f(self._h, _ptr(ref_ids), _ptr(y), B, int(half_window), _ptr(lag), _ptr(mag),
                                         _stream(stream)))
        return lag, mag

    def reset_references(self):
        _raise(lib().sidwt_reset_references(self._h))

    def set_timing(self, on: bool = True):
        _raise(lib().sidwt_set_timing(self._h, 1 if on else 0))

    def read_timing(self, reset: bool = True) -> dict:
        t = Timing()
        _raise(lib().sidwt_read_timing(self._h, ctypes.byref(t), 1 if reset else 0))
        return t.as_dict()


def correlate_static(filter, N: int, J: int, x: torch.Tensor, y: torch.Tensor, lag: torch.Tensor,
                     mag: torch.Tensor, norm: torch.Tensor, stream=None):
    """Allocation-free correlation of the pulses y against one stored signal x
    (sidwt_correlate_static): the library uses its fixed static scratch array
    and writes the peaks into the caller's lag / mag / norm [B, J+1] tensors."""
    B = y.shape[0]
    _raise(lib().sidwt_correlate_static(_filter_id(filter), int(N), int(J), _ptr(x), _ptr(y), B, _ptr(lag),
                                        _ptr(mag), _ptr(norm), _stream(stream)))


class Ragged:
    """Pulses of uneven length, depth and filter, each against its own stored
    signal, correlated in one persistent launch (sidwt_ragged_*)."""

    def __init__(self):
        h = _vp()
        _raise(lib().sidwt_ragged_create(ctypes.byref(h)))
        self._h = h
        self.refs = []  # (filter, N, J) per stored reference
        self._layout = None

    def close(self):
        if getattr(self, "_h", None):
            lib().sidwt_ragged_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reserve(self, tree_elems: int, pyr_elems: int, slots: int):
        _raise(lib().sidwt_ragged_reserve(self._h, tree_elems, pyr_elems, slots))

    def set_precision(self, precision):
        """'fp32' (default) or 'bf16x3': applies to later stores and correlations."""
        _raise(lib().sidwt_ragged_set_precision(self._h, _prec_id(precision)))

    def check(self, stream=None):
        _raise(lib().sidwt_ragged_check(self._h, _stream(stream)))

    def store_reference(self, filter, N: int, J: int, x: torch.Tensor, stream=None) -> int:
        if x.dtype != torch.complex64 or not x.is_cuda or x.numel() != N or not x.is_contiguous():
            raise ValueError("reference must be a contiguous CUDA complex64 tensor of N samples")
        rid = _i32(-1)
        _raise(lib().sidwt_ragged_store_reference(self._h, _filter_id(filter), int(N), int(J), _ptr(x),
                                                  ctypes.byref(rid), _stream(stream)))
        self.refs.append((_filter_id(filter), int(N), int(J)))
        return rid.value

    def store_references(self, filters, Ns, Js, x: torch.Tensor, offsets, stream=None) -> list[int]:
        """Store many signals at once (sidwt_ragged_store_references): item i
        is x[offsets[i]:offsets[i] + Ns[i]] (x a packed CUDA complex64 buffer)."""
        if x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("signals must be a contiguous CUDA complex64 buffer")
        f = np.ascontiguousarray([_filter_id(v) for v in filters], dtype=np.int32)
        n = np.ascontiguousarray(Ns, dtype=np.int64)
        j = np.ascontiguousarray(Js, dtype=np.int32)
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        if not (f.shape == n.shape == j.shape == off.shape):
            raise ValueError("one filter, N, J and offset per item")
        ids = np.zeros(f.shape, dtype=np.int32)
        _raise(lib().sidwt_ragged_store_references(self._h, f.size, f.ctypes.data, n.ctypes.data, j.ctypes.data,
                                                   _ptr(x), off.ctypes.data, x.numel(), ids.ctypes.data,
                                                   _stream(stream)))
        self.refs.extend((int(a), int(b), int(c)) for a, b, c in zip(f, n, j))
        return ids.tolist()

    def slots_of(self, ref_ids) -> tuple[np.ndarray, int]:
        """First peak slot of every item and the total slot count."""
        js = np.array([self.refs[int(r)][2] for r in ref_ids], dtype=np.int64)
        first = np.concatenate([[0], np.cumsum(js + 1)[:-1]]) if len(js) else np.zeros(0, np.int64)
        return first, int((js + 1).sum())

    def _args(self, ref_ids, offsets):
        ids = np.ascontiguousarray(np.asarray(ref_ids, dtype=np.int32))
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        if ids.shape != off.shape:
            raise ValueError("one offset per item")
        return ids, off

    def correlate(self, ref_ids, offsets, y: torch.Tensor, stream=None) -> int:
        """y: packed complex64 CUDA buffer; returns the number of peak slots."""
        ids, off = self._args(ref_ids, offsets)
        _raise(lib().sidwt_ragged_correlate(self._h, ids.size, ids.ctypes.data, off.ctypes.data, _ptr(y),
                                            y.numel(), _stream(stream)))
        self._layout = ids
        return self.slots_of(ids)[1]

    def set_split(self, mode):
        """Contraction splitting of the tensor-core tiles (sidwt_ragged_set_split):
        "auto" (0), "never" (1) or "always" (2)."""
        m = {"auto": 0, "never": 1, "always": 2}.get(mode, mode)
        _raise(lib().sidwt_ragged_set_split(self._h, int(m)))

    def r_rows_of(self, ref_ids) -> tuple[np.ndarray, int]:
        """First element of every item's J + 1 rows of N lags in the r output, and the total."""
        sz = np.array([(self.refs[int(r)][2] + 1) * self.refs[int(r)][1] for r in ref_ids], dtype=np.int64)
        first = np.concatenate([[0], np.cumsum(sz)[:-1]]) if len(sz) else np.zeros(0, np.int64)
        return first, int(sz.sum())

    def correlate_r(self, ref_ids, offsets, y: torch.Tensor, stream=None):
        """As correlate, and the correlation at every lag and scale
        (sidwt_ragged_correlate_r): returns (slots, r) with r a packed complex64
        tensor; item i's scale j is r[first[i] + j N_i : + N_i] (r_rows_of)."""
        ids, off = self._args(ref_ids, offsets)
        _, total = self.r_rows_of(ids)
        r = torch.zeros(max(1, total), dtype=torch.complex64, device=y.device)
        _raise(lib().sidwt_ragged_correlate_r(self._h, ids.size, ids.ctypes.data, off.ctypes.data, _ptr(y),
                                              y.numel(), _ptr(r), r.numel(), _stream(stream)))
        self._layout = ids
        return self.slots_of(ids)[1], r[:total]

    def graph_create(self, ref_ids, offsets, y: torch.Tensor) -> int:
        ids, off = self._args(ref_ids, offsets)
        n = _i32(0)
        _raise(lib().sidwt_ragged_graph_create(self._h, ids.size, ids.ctypes.data, off.ctypes.data, _ptr(y),
                                               y.numel(), ctypes.byref(n)))
        self._graph_layout = ids
        return n.value

    def graph_launch(self, stream=None) -> int:
        _raise(lib().sidwt_ragged_graph_launch(self._h, _stream(stream)))
        self._layout = self._graph_layout
        return self.slots_of(self._layout)[1]

    def peaks(self, n_slots: int, stream=None):
        dev = torch.cuda.current_device()
        lag = torch.empty(n_slots, dtype=torch.int32, device=dev)
        mag = torch.empty(n_slots, dtype=torch.float32, device=dev)
        norm = torch.empty(n_slots, dtype=torch.float64, device=dev)
        _raise(lib().sidwt_ragged_peaks(self._h, n_slots, _ptr(lag), _ptr(mag), _ptr(norm), _stream(stream)))
        return lag, mag, norm

    def peaks_into(self, n_slots: int, lag, mag, norm, stream=None):
        _raise(lib().sidwt_ragged_peaks(self._h, n_slots, _ptr(lag), _ptr(mag), _ptr(norm), _stream(stream)))

    def autotune(self, cache_path: str | None = None, stream=None):
        _raise(lib().sidwt_ragged_autotune(self._h, cache_path.encode() if cache_path else None, _stream(stream)))

    def tuning(self) -> np.ndarray:
        out = np.zeros(32, np.int32)
        _raise(lib().sidwt_ragged_tuning(self._h, out.ctypes.data))
        return out

    def tc_weights(self) -> np.ndarray:
        """[4, 25]: cost weight of tile width 256 / 128 / 64 / 192 by log2 band length."""
        out = np.zeros((4, 25), np.float32)
        _raise(lib().sidwt_ragged_tc_weights(self._h, out.ctypes.data))
        return out

    def set_timing(self, on: bool = True):
        _raise(lib().sidwt_ragged_set_timing(self._h, 1 if on else 0))

    def read_timing(self, reset: bool = True) -> dict:
        t = Timing()
        _raise(lib().sidwt_ragged_read_timing(self._h, ctypes.byref(t), 1 if reset else 0))
        return t.as_dict()

    def reset_references(self):
        _raise(lib().sidwt_ragged_reset_references(self._h))
        self.refs = []


class Server:
    """Continuous-batching request loop (sidwt_server_*)."""

    def __init__(self, lanes=4, max_batch=64, max_j=10, memory_cap_bytes=40 << 30, max_lane_samples=1 << 22,
                 precision="fp32"):
        cfg = ServerConfig(lanes, max_batch, max_j, memory_cap_bytes, max_lane_samples, _prec_id(precision))
        h = _vp()
        _raise(lib().sidwt_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.max_j = max_j
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().sidwt_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def add_waveform(self, x: np.ndarray) -> int:
        x = np.ascontiguousarray(np.asarray(x, dtype=np.complex64))
        wid = _i32(-1)
        _raise(lib().sidwt_server_add_waveform(self._h, x.ctypes.data, x.size, ctypes.byref(wid)))
        return wid.value

    def start(self):
        _raise(lib().sidwt_server_start(self._h))

    def submit(self, wave: int, filter, N: int, J: int, y: torch.Tensor) -> int:
        """y: host complex64 tensor of N samples (pinned is fastest); kept alive until finished."""
        if y.is_cuda or y.dtype != torch.complex64 or y.numel() != N or not y.is_contiguous():
            raise ValueError("y must be a contiguous host complex64 tensor of N samples")
        rid = _i64(-1)
        _raise(lib().sidwt_server_submit(self._h, wave, _filter_id(filter), int(N), int(J), _ptr(y),
                                         ctypes.byref(rid)))
        self._keep[rid.value] = (y, J)
        return rid.value

    def wait(self, rid: int, timeout_s: float = 30.0):
        _raise(lib().sidwt_server_wait(self._h, rid, timeout_s))

    def drain(self, timeout_s: float = 60.0):
        _raise(lib().sidwt_server_drain(self._h, timeout_s))

    def result(self, rid: int):
        J = self._keep[rid][1]
        lag = np.zeros(J + 1, np.int32)
        mag = np.zeros(J + 1, np.float32)
        norm = np.zeros(J + 1, np.float64)
        lat = ctypes.c_double(0.0)
        _raise(lib().sidwt_server_result(self._h, rid, lag.ctypes.data, mag.ctypes.data, norm.ctypes.data,
                                         ctypes.byref(lat)))
        return lag, mag, norm, lat.value

    def forget(self, rid: int):
        _raise(lib().sidwt_server_forget(self._h, rid))
        self._keep.pop(rid, None)

    def stats(self, reset: bool = False) -> dict:
        st = ServerStats()
        _raise(lib().sidwt_server_read_stats(self._h, ctypes.byref(st), 1 if reset else 0))
        return st.as_dict()


def tc_selftest(stream=None):
    """Run the tensor-core layout self-test; returns (out [128, 64] float32, err flag)."""
    dev = torch.cuda.current_device()
    out = torch.zeros((128, 64), dtype=torch.float32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    _raise(lib().sidwt_tc_selftest(_ptr(out), _ptr(err), _stream(stream)))
    return out, err


STALL_ANALYSIS = 1      # the pipelined received analysis issues no input copy
STALL_TC_SELFTEST = 2   # sidwt_tc_selftest issues no MMA


def debug_stall(what: int):
    """Test hook (sidwt_debug_stall): make the named bounded device waits run
    out on purpose (0 restores normal operation).  Process-wide."""
    _raise(lib().sidwt_debug_stall(int(what)))


def level_slices(N: int, J: int, l: int) -> tuple[slice, slice]:
    """(c_l, d_l) element slices of a received pyramid row."""
    K = N >> l
    off = 2 * N - 4 * K
    return slice(off, off + K), slice(off + K, off + 2 * K)


def as_numpy_complex(t: torch.Tensor) -> np.ndarray:
    """complex64 tensor, or int32 pairs [..., 2], as complex128 numpy."""
    a = t.detach().cpu()
    if a.dtype == torch.complex64:
        return a.numpy().astype(np.complex128)
    a = a.numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def synthesize(filter, lo: torch.Tensor, hi: torch.Tensor, stream=None) -> torch.Tensor:
    """Eq. 21 (sidwt_synthesize): c_{l-1} [B][2H] from the bands lo, hi [B][H]
    (complex64 CUDA tensors whose rows may be strided views of one buffer)."""
    if lo.dim() == 1:
        lo, hi = lo[None], hi[None]
    B, H = lo.shape
    if lo.dtype != torch.complex64 or hi.dtype != torch.complex64 or lo.stride(1) != 1 or hi.stride(1) != 1 or \
            lo.stride(0) != hi.stride(0):
        raise ValueError("lo and hi: complex64 rows with unit inner stride and the same row stride")
    out = torch.empty((B, 2 * H), dtype=torch.complex64, device=lo.device)
    _raise(lib().sidwt_synthesize(_filter_id(filter), H, B, _ptr(lo), _ptr(hi), lo.stride(0) if B > 1 else H,
                                  _ptr(out), _stream(stream)))
    return out


def detect(r: torch.Tensor, threshold_db: float = 10.0, max_det: int = 32, stream=None):
    """Per-row detections (sidwt_detect) of complex64 correlations r[..., N]:
    (count [...], lag [..., max_det], mag [..., max_det])."""
    if r.dtype != torch.complex64 or not r.is_cuda or not r.is_contiguous():
        raise ValueError("r must be a contiguous CUDA complex64 tensor")
    lead = tuple(r.shape[:-1])
    N = r.shape[-1]
    rows = int(np.prod(lead)) if lead else 1
    count = torch.empty(lead, dtype=torch.int32, device=r.device)
    lag = torch.full(lead + (max_det,), -1, dtype=torch.int32, device=r.device)
    mag = torch.zeros(lead + (max_det,), dtype=torch.float32, device=r.device)
    _raise(lib().sidwt_detect(_ptr(r), rows, N, float(threshold_db), int(max_det), _ptr(count), _ptr(lag), _ptr(mag),
                              _stream(stream)))
    return count, lag, mag
