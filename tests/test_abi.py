"""The C-ABI library builds, loads, and exports every entry point that
include/m2nufft.h declares (no GPU needed: nothing is computed here)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2407_01943_gb300 as pkg
from paper_2407_01943_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "m2nufft.h")


def declared_functions(header=HEADER, prefix="m2nufft_"):
    src = open(header).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(" + prefix + r"\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["m2nufft_plan", "m2nufft_exec", "m2nufft_destroy", "m2nufft_exec_batch",
              "m2nufft_get_tapers", "m2nufft_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    path = pkg.build()
    lib = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (m2nufft_\w+)", out))
    assert set(declared_functions()) <= exported
    # the binding wraps exactly the declared set
    assert sorted(n for n, _, _ in binding.EXPORTS) == declared_functions()


def test_version_string_without_gpu():
    assert "sm_103a" in binding.version()


def test_batch_argument_errors_without_gpu():
    """The uneven-batch entry points reject bad arguments before any device work, with the
    documented status and a message naming the entry point (an empty batch is a no-op)."""
    lib = binding.load()
    VP = ctypes.c_void_p
    none = ctypes.POINTER(VP)()
    assert lib.m2nufft_exec_batch(none, none, 0, none, none, none, None) == 0
    assert lib.m2nufft_exec_batch(none, none, -1, none, none, none, None) == 1
    assert b"m2nufft_exec_batch" in lib.m2nufft_last_error()
    # the F entry point requires the Fs array itself, even for an empty batch
    assert lib.m2nufft_exec_batch_ftest(none, none, 0, none, none, none, none, None) == 1
    assert b"Fs is NULL" in lib.m2nufft_last_error()
    fs = (VP * 1)(None)
    assert lib.m2nufft_exec_batch_ftest(none, none, 0, none, none, none, fs, None) == 0
    assert lib.m2nufft_exec_batch_ftest(none, none, -2, none, none, none, fs, None) == 1
    assert b"m2nufft_exec_batch_ftest" in lib.m2nufft_last_error()
    # a NULL plan inside a non-empty batch is named by its index
    plans = (VP * 2)(None, None)
    xs = (VP * 2)(None, None)
    assert lib.m2nufft_exec_batch(plans, xs, 2, none, none, none, None) == 1
    assert b"plan or x 0 is NULL" in lib.m2nufft_last_error()


def test_struct_layouts_match_header():
    # m2_fgrid: 2 doubles + int64; m2_opts: int, double, size_t, int, int, int (natural alignment)
    assert ctypes.sizeof(binding.m2_fgrid) == 24
    assert ctypes.sizeof(binding.m2_opts) == 56
    assert binding.m2_opts.sigma.offset == 40 and binding.m2_opts.tune.offset == 48
    assert binding.m2_opts.path.offset == 32 and binding.m2_opts.tapers.offset == 36
    assert binding.m2_opts.tol.offset == 8 and binding.m2_opts.mem_budget.offset == 16


def test_server_header_exports():
    hdr = os.path.join(ROOT, "include", "m2serve.h")
    names = declared_functions(hdr, "m2serve_")
    assert names == sorted(n for n, _, _ in binding.SERVE_EXPORTS)
    lib = ctypes.CDLL(pkg.build())
    for n in names:
        assert hasattr(lib, n), n


def test_info_layout_matches_c_compiler(tmp_path):
    """m2_info as the C compiler lays it out from the header equals the binding's ctypes mirror."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "info.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "m2nufft.h"\n'
                   'int main(void) { printf("%zu %zu %zu\\n", sizeof(m2_info), offsetof(m2_info, gep_seconds),'
                   ' offsetof(m2_info, spread_entries)); return 0; }\n')
    exe = tmp_path / "info"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    size, gep, ent = (int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                                      check=True).stdout.split())
    assert ctypes.sizeof(binding.m2_info) == size
    assert binding.m2_info.gep_seconds.offset == gep
    assert binding.m2_info.spread_entries.offset == ent
