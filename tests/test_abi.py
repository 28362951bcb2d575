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
    assert ctypes.sizeof(_ffi.MultStats) == 14 * 8
    assert ctypes.sizeof(_ffi.SignOpts) == 8 + 8 + 4 + 4 + 8 + 8 + 4 + 4 + 4 + 4
    # 4 int32, 5 double, int64, 2 double, int64, then the histories
    assert _ffi.SignReport.residual_history.offset == 16 + 40 + 8 + 16 + 8
    assert _ffi.SignReport.ms_symbolic.offset == _ffi.SignReport.nnzb_history.offset + 8 * _ffi.MAX_HISTORY


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """sizeof / offsetof of every ABI struct, from gcc reading the header, equal the ctypes mirrors."""
    import shutil
    import subprocess
    from paper_2003_03868_gb300 import _ffi
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    probes = {
        "dbcsr_mult_stats": (_ffi.MultStats, ["flops", "dev2_filtered", "ms_filter", "bytes_min", "n_launches",
                                               "flops_tensor", "bytes_tensor", "n_tiles"]),
        "dbcsr_sign_opts": (_ffi.SignOpts, ["switch_tol", "verbose", "flags", "order", "reserved"]),
        "dbcsr_sign_report": (_ffi.SignReport, ["alpha", "n_products", "residual_history", "nnzb_history",
                                               "ms_symbolic", "ms_low", "flops_low", "bytes_min_fp64",
                                               "launches_fp64", "flops_tensor", "bytes_tensor"]),
        "dbcsr_kernel_cfg": (_ffi.KernelCfg, ["prefetch2", "split"]),
        "dbcsr_tune_record": (_ffi.TuneRecord, ["cfg", "ms", "gflops"]),
        "dbcsr_mlp_opts": (_ffi.MlpOpts, ["lr", "eps"]),
        "dbcsr_mlp_report": (_ffi.MlpReport, [f[0] for f in _ffi.MlpReport._fields_]),
    }
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dbcsr_gb.h"', "int main(void) {"]
    for t, (_, fields) in probes.items():
        lines.append(f'  printf("{t} %zu\\n", sizeof({t}));')
        for f in fields:
            lines.append(f'  printf("{t}.{f} %zu\\n", offsetof({t}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines())
    for t, (cls, fields) in probes.items():
        assert int(got[t]) == ctypes.sizeof(cls), t
        for f in fields:
            assert int(got[f"{t}.{f}"]) == getattr(cls, f).offset, f"{t}.{f}"
