"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/henn.h declares; the ctypes structs match the C layouts.
No compute call is made (no GPU needed)."""
from __future__ import annotations

import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "henn.h")


@pytest.fixture(scope="module")
def lib_path():
    from paper_2505_17368_gb300.build import build

    return build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(henn_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    fns = declared_functions()
    for f in ["henn_build", "henn_search", "henn_free", "henn_last_error"]:
        assert f in fns


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    lib = C.CDLL(lib_path)
    for f in declared_functions():
        getattr(lib, f)


def test_binding_lists_every_export(lib_path):
    from paper_2505_17368_gb300 import binding

    assert sorted(binding.EXPORTS) == declared_functions()


def test_struct_layouts_match_c():
    from paper_2505_17368_gb300 import binding

    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "henn.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(henn_build_params), offsetof(henn_build_params, seed),
         offsetof(henn_build_params, sampler),
         sizeof(henn_search_params), offsetof(henn_search_params, ef_upper),
         offsetof(henn_search_params, time_kernel),
         sizeof(henn_index_info), offsetof(henn_index_info, build_seconds),
         offsetof(henn_index_info, graph_updates), sizeof(henn_serve_params),
         offsetof(henn_serve_params, exact_upper));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "s.c")
        exe = os.path.join(td, "s")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    want = [C.sizeof(binding.BuildParams), binding.BuildParams.seed.offset, binding.BuildParams.sampler.offset,
            C.sizeof(binding.SearchParams),
            binding.SearchParams.ef_upper.offset, binding.SearchParams.time_kernel.offset, C.sizeof(binding.IndexInfo),
            binding.IndexInfo.build_seconds.offset, binding.IndexInfo.graph_updates.offset,
            C.sizeof(binding.ServeParams), binding.ServeParams.exact_upper.offset]
    assert got == want


def test_missing_library_fails_loudly(tmp_path):
    from paper_2505_17368_gb300 import binding

    with pytest.raises(ImportError):
        binding._lib = None
        try:
            binding.load(str(tmp_path / "nope.so"))
        finally:
            binding._lib = None
