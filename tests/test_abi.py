"""The C-ABI library builds, loads and exports every function include/ffp.h
declares; its host-only entry points behave without a GPU (no compute)."""
import ctypes
import os
import re

import pytest

from paper_1909_09771_gb300 import build as B
from paper_1909_09771_gb300 import ffp

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ffp.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ffp.load()


def test_exports_every_declared_symbol(lib):
    names = ffp.declared_functions()
    assert {"ffp_setup", "ffp_apply", "ffp_pcg_solve", "ffp_spmv", "ffp_workspace_bytes",
            "ffp_destroy", "ffp_strerror", "ffp_export"} <= set(names)
    raw = ctypes.CDLL(ffp.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), f"{n} declared in include/ffp.h but not exported"


def test_header_constants_match_binding():
    txt = open(HDR).read()
    defs = dict(re.findall(r"#define\s+(FFP_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", txt))
    for k, v in defs.items():
        if hasattr(ffp, k):
            assert getattr(ffp, k) == int(v), k


def test_workspace_bytes_host_only(lib):
    assert ffp.workspace_bytes((32, 32, 32), "fp64") > 32 ** 3 * 8 * 12
    assert ffp.workspace_bytes((32, 32, 32), "fp32") < ffp.workspace_bytes((32, 32, 32), "fp64")
    g = ffp.Grid(0, 4, 4, 1, 1, 1)
    assert lib.ffp_workspace_bytes(ctypes.byref(g), 0) == 0
    g = ffp.Grid(ffp.FFP_MAX_NX + 1, 2, 2, 1, 1, 1)
    assert lib.ffp_workspace_bytes(ctypes.byref(g), 0) == 0
    g = ffp.Grid(4, 4, 4, 1, 1, 1)
    assert lib.ffp_workspace_bytes(ctypes.byref(g), 7) == 0


def test_net_workspace_bytes_host_only(lib):
    """The network's padded BF16 layout: two 16-byte planes per padded cell and
    batch, with guards; rows longer than FFP_NET_MAX_NX cells are rejected."""
    f = lib.ffp_net_workspace_bytes
    f.restype = ctypes.c_size_t
    g = ffp.Grid(64, 64, 64, 1, 1, 1)
    inf, trn = f(ctypes.byref(g), 1, 0), f(ctypes.byref(g), 1, 1)
    padded = 66 ** 3 * 32
    assert 2 * padded <= inf < 3 * padded and 7 * padded <= trn < 8 * padded + (64 << 20)
    g = ffp.Grid(ffp.FFP_NET_MAX_NX + 1, 2, 2, 1, 1, 1)
    assert f(ctypes.byref(g), 1, 0) == 0
    g = ffp.Grid(4, 4, 4, 1, 1, 1)
    assert f(ctypes.byref(g), 0, 0) == 0


def test_strerror_and_null_args(lib):
    assert lib.ffp_strerror(0) == b"ok"
    assert b"breakdown" in lib.ffp_strerror(ffp.FFP_ERR_BREAKDOWN)
    # argument checks happen before any CUDA call
    assert lib.ffp_apply(None, None, None, None) == ffp.FFP_ERR_ARG
    assert lib.ffp_spmv(None, None, None, None) == ffp.FFP_ERR_ARG
    h = ctypes.c_void_p()
    g = ffp.Grid(4, 4, 4, 1, 1, 1)
    assert lib.ffp_setup(ctypes.byref(g), None, None, 0, None, 0, 0, None, 0, None,
                         ctypes.byref(h)) == ffp.FFP_ERR_ARG


def test_struct_layouts_match_binding(tmp_path):
    """The ctypes mirrors of ffp_grid, ffp_bc, ffp_stats and ffp_batch_config
    have the size and field offsets a C compiler gives the structs of
    include/ffp.h (a mismatch would corrupt every call that passes them)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    mirrors = {"ffp_grid": ffp.Grid, "ffp_bc": ffp.BC, "ffp_stats": ffp.Stats,
               "ffp_batch_config": ffp.BatchConfig}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HDR}"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
