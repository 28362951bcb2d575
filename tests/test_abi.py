"""The C-ABI library builds, loads and exports every entry point its header declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dbcsr_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2003_03868_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = _declared("dbcsr_gb.h") + _declared("dbcsr_gb_bench.h")
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2003_03868_gb300 import _ffi
    bound = {n for n, _, _ in _ffi.SIGNATURES}
    assert set(_declared("dbcsr_gb.h")) | set(_declared("dbcsr_gb_bench.h")) <= bound


def test_version_and_error_string_without_gpu(libpath):
    import paper_2003_03868_gb300 as gb
    assert b"sm_103a" in gb.lib().dbcsr_version()
    # a call on a null handle fails cleanly and sets the error string (no GPU touched)
    st = gb.lib().dbcsr_finalize(None)
    assert st == 1
    assert b"null" in gb.lib().dbcsr_last_error()


def test_struct_layouts_match_header():
    from paper_2003_03868_gb300 import _ffi
    assert ctypes.sizeof(_ffi.MultStats) == 9 * 8
    assert ctypes.sizeof(_ffi.SignOpts) == 8 + 8 + 4 + 4 + 8 + 8 + 4 + 4
    # 4 int32, 5 double, int64, 2 double, int64, then the histories
    assert _ffi.SignReport.residual_history.offset == 16 + 40 + 8 + 16 + 8
