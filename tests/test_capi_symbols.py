"""The C-ABI library builds, loads without a GPU, and exports every function
that include/plse.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "plse.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(plse_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_10453_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("plse_create", "plse_solve", "plse_destroy", "plse_local_search",
                 "plse_pop_update", "plse_matching", "plse_crossover", "plse_distances"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_2103_10453_gb300 import plse
    assert sorted(plse.SIGNATURES) == declared_functions()


def test_strerror_and_invalid_arguments_without_gpu(lib):
    lib.plse_strerror.restype = ctypes.c_char_p
    assert lib.plse_strerror(0) == b"success"
    assert lib.plse_strerror(-1) == b"invalid argument"
    h = ctypes.c_void_p()
    assert lib.plse_create(0, None, ctypes.byref(h)) == -1          # rejected before any CUDA call
    assert lib.plse_create(200, None, ctypes.byref(h)) == -1
    empty128 = (ctypes.c_int8 * (128 * 128))()                      # a valid grid one order too large
    assert lib.plse_create(128, empty128, ctypes.byref(h)) == -1


def test_binding_structs_match_the_header_layout(tmp_path):
    """sizeof / offsetof of every struct in include/plse.h, as gcc lays it out,
    equal the ctypes mirrors of the binding."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2103_10453_gb300 import plse
    structs = {"plse_params": plse.Params, "plse_walk_stats": plse.WalkStats,
               "plse_solve_stats": plse.SolveStats, "plse_job": plse.Job, "plse_result": plse.Result}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "plse.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for cname, cls in structs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(cls, f).offset, (cname, f)
