"""The C ABI library loads and exports every entry point that include/*.h
declares, and the ctypes structures match the C layouts (no GPU needed)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_2105_11788_gb300 import _build, bisim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[\w\s\*]*?\b(bisim_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return bisim.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "bisim_plan" in names and "bisim_refine" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    for name in bisim.EXPORTED:
        assert name in names


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "bisim.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(bisim_opts),"
        " sizeof(bisim_stats), offsetof(bisim_opts, round_cap), offsetof(bisim_stats, t_plan_ms),"
        " offsetof(bisim_stats, engine), offsetof(bisim_opts, max_ctas)); return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(bisim.bisim_opts), ctypes.sizeof(bisim.bisim_stats),
            bisim.bisim_opts.round_cap.offset, bisim.bisim_stats.t_plan_ms.offset,
            bisim.bisim_stats.engine.offset, bisim.bisim_opts.max_ctas.offset]
    assert got == want


def test_error_strings_and_version(lib):
    assert bisim.bisim_version() >= 100
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert bisim.strerror(code)
    assert bisim.strerror(-5) == "grid barrier wait timed out"


def test_null_arguments_rejected_without_device(lib):
    # argument checks happen before any CUDA call
    rc = lib.bisim_plan(-1, 0, 1, None, None, None, None, None, None, ctypes.byref(ctypes.c_void_p()))
    assert rc == bisim.BISIM_EINVAL
    rc = lib.bisim_plan(3, 2, 0, None, None, None, None, None, None, ctypes.byref(ctypes.c_void_p()))
    assert rc == bisim.BISIM_EINVAL
    rc = lib.bisim_refine(None, None, None)
    assert rc == bisim.BISIM_EINVAL
    lib.bisim_plan_destroy(None)


def test_library_does_not_link_the_oracle(lib):
    out = subprocess.check_output(["nm", "-D", _build.LIB]).decode()
    assert "oracle_" not in out
