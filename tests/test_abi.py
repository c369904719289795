"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads,
exports every entry point include/sidwt.h declares, and rejects bad plan
arguments before touching a GPU."""
import ctypes
import re
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    text = (ROOT / "include" / "sidwt.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sidwt_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_cs_0607001_gb300 import build, sidwt
    build.build()
    return sidwt.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("sidwt_plan_create", "sidwt_store_reference", "sidwt_correlate", "sidwt_peaks", "sidwt_analyze"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_cs_0607001_gb300 import sidwt
    out = subprocess.run(["nm", "-D", "--defined-only", str(sidwt.library_path())], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_library_is_built_for_sm_103a(lib):
    from paper_cs_0607001_gb300 import build, sidwt
    assert "sm_103a" in sidwt.version()
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_bad_plan_arguments_are_rejected_on_the_host(lib):
    h = ctypes.c_void_p()
    assert lib.sidwt_plan_create(1, 1000, 4, ctypes.byref(h)) == 1  # 1000 % 16 != 0
    assert b"multiple" in lib.sidwt_last_error()
    assert lib.sidwt_plan_create(7, 1024, 4, ctypes.byref(h)) == 1  # unknown filter
    assert lib.sidwt_plan_create(1, 1024, 0, ctypes.byref(h)) == 1  # J < 1
    assert lib.sidwt_plan_create(1, 1 << 20, 16, ctypes.byref(h)) == 1  # J > 15
    assert lib.sidwt_plan_create(1, 1024, 4, None) == 1
    assert lib.sidwt_correlate(None, None, None, 0, 0, None, None) == 1
    assert lib.sidwt_plan_destroy(None) == 0


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    from paper_cs_0607001_gb300 import build, sidwt
    monkeypatch.setattr(sidwt, "_lib", None)
    monkeypatch.setattr(build, "LIB", tmp_path / "missing.so")
    with pytest.raises(RuntimeError, match="not built"):
        sidwt.lib()


def test_debug_stall_takes_only_known_flags(lib):
    """The test hook that makes bounded device waits run out is host state
    only: unknown bits are rejected, 0 restores normal operation."""
    assert lib.sidwt_debug_stall(4) == 1
    assert b"unknown flag" in lib.sidwt_last_error()
    assert lib.sidwt_debug_stall(3) == 0
    assert lib.sidwt_debug_stall(0) == 0
