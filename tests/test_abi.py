"""CPU-only checks of the C ABI: the library builds for sm_103a, loads, exports
every function declared in include/tb.h, and its tb_params layout matches the
ctypes mirror (compiled C probe of sizeof/offsetof).  No compute calls."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tb.h")


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_4497_gb300 import binding
    return binding


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:tb_status|const char\s*\*)\s*(tb_\w+)\s*\(", src, re.M)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for need in ("tb_build_neighbors", "tb_assemble_H", "tb_krylov_density", "tb_find_mu",
                 "tb_forces", "tb_md_step"):
        assert need in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(built.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", built.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (tb_\w+)", out))
    assert set(declared_functions()) <= exported


def test_build_flags_target_sm103a(built):
    from paper_0910_4497_gb300 import build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_params_struct_layout_matches_c(built):
    fields = [f[0] for f in built.TBParams._fields_]
    body = "\n".join(
        f'printf("%s %zu\\n", "{f}", offsetof(tb_params, {f}));' for f in fields)
    prog = f"""#include <stdio.h>
#include <stddef.h>
#include "tb.h"
int main(void) {{ printf("size %zu\\n", sizeof(tb_params)); {body} return 0; }}"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = dict(line.split() for line in out.strip().splitlines())
    assert int(got["size"]) == ctypes.sizeof(built.TBParams)
    for f in fields:
        assert int(got[f]) == getattr(built.TBParams, f).offset, f


def test_params_default_without_gpu(built):
    p = built.TBParams()
    assert built.lib().tb_params_default(ctypes.byref(p)) == 0
    assert p.kT == 0.1 and p.r == 8 and p.max_hnbr == 32
    assert p.group_m == 1 and p.max_union == 0
    assert built.lib().tb_params_default(None) == 1
