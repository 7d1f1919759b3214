"""CPU checks of the C-ABI boundary: the library builds, loads without a GPU,
and exports every function include/tcprod.h declares; the binding's structs
match the header's sizes."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2103_11847_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(?:int|const char\*|void)\s+(tc_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    path = B.lib_path()
    if not os.path.exists(path):
        B.build()
    return path


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["tc_plan_create", "tc_plan_destroy", "tc_cprod", "tc_cprod_adjoint",
                     "tc_gkb_init", "tc_gkb_step", "tc_lsqr_c", "tc_gmres_c",
                     "tc_tikhonov_gcv"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_string_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.tc_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.tc_version()


def _c_layout(tmp_path, struct, fields):
    """sizeof and offsetof of a header struct, from the host C compiler."""
    gcc = shutil.which("gcc") or shutil.which("cc")
    if not gcc:
        pytest.skip("no host C compiler")
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tcprod.h"', 'int main(void) {',
             f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ['  return 0;', '}']
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


def test_binding_structs_match_header(tmp_path):
    from paper_2103_11847_gb300 import tcprod
    for cls, struct in ((tcprod.tc_opts, "tc_opts"), (tcprod.tc_solve_info, "tc_solve_info")):
        names = [f[0] for f in cls._fields_]
        cnames = ["lambda" if n == "lambda_" else n for n in names]
        size, offs = _c_layout(tmp_path, struct, cnames)
        assert ctypes.sizeof(cls) == size, struct
        assert [getattr(cls, n).offset for n in names] == offs, struct
    assert set(tcprod._SIGS) == set(declared_functions())


def test_invalid_arguments_rejected_on_host(libpath):
    # Host-side argument checks return TC_EINVAL before any CUDA call.
    lib = ctypes.CDLL(libpath)
    lib.tc_plan_create.restype = ctypes.c_int
    h = ctypes.c_void_p()
    assert lib.tc_plan_create(ctypes.byref(h), 0, 4, 4, 3, ctypes.c_void_p(16), None, None,
                              None) == -1
    assert lib.tc_plan_create(None, 4, 4, 4, 3, ctypes.c_void_p(16), None, None, None) == -1
    assert lib.tc_cprod(None, None, None, None) == -1
    lib.tc_lsqr_c.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int, ctypes.c_double,
                                                      ctypes.c_double] + [ctypes.c_void_p] * 3
    assert lib.tc_lsqr_c(None, None, None, None, 10, 0.0, -1.0, None, None, None) == -1
