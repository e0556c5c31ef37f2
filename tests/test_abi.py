"""The C-ABI library builds, loads without a GPU, and exports every entry point gb.h declares."""
import ctypes
import os
import re

import pytest

from paper_2307_03763_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gb_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_the_four_calls_and_context():
    names = declared_functions()
    for n in ("gb_waveform", "gb_loglik", "gb_loglik_grad", "gb_mh_independence", "gb_ctx_create",
              "gb_ctx_destroy", "gb_last_error", "gb_ctx_check"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2307_03763_gb300 import api
    assert set(api._SIGNATURES) == set(declared_functions())


def test_window_struct_layout():
    from paper_2307_03763_gb300 import api
    assert ctypes.sizeof(api.Window) == 40
    assert ctypes.sizeof(api.Obs) == 24


def test_header_is_plain_c_and_links(libpath, tmp_path):
    # a C99 program that takes the address of every declared entry point
    # compiles without warnings against gb.h and links against the library
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = declared_functions()
    src = tmp_path / "use_gb.c"
    src.write_text('#include "gb.h"\n#include <stdio.h>\nint main(void) {\n'
                   + "".join('    printf("%%p\\n", (void*)&%s);\n' % n for n in names)
                   + "    return 0;\n}\n")
    exe = tmp_path / "use_gb"
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I",
           os.path.join(ROOT, "include"), str(src), "-o", str(exe), libpath,
           "-Wl,-rpath," + os.path.dirname(libpath)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
