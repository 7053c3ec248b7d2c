"""The C-ABI library builds, loads and exports every symbol include/stencil.h
declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"STENCIL_API\s+[\w\s\*]+?\b(\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2310_01882_b300 import build, stencil
    build.build()
    return stencil.lib()


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("stencil_jacobi_sweep", "stencil_residual", "stencil_advect_uvw", "stencil_ctx_create"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2310_01882_b300 import stencil
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in stencil.SIGNATURES, name


def test_host_side_validation_without_gpu(lib):
    """A null context is rejected before any CUDA call."""
    from paper_2310_01882_b300 import stencil
    g = stencil.stencil_grid(None, 4, 4, 4, 6, 36, 0, 0)
    rc = lib.stencil_jacobi_sweep(None, ctypes.byref(g), ctypes.byref(g), ctypes.byref(g), None, 0.1, 1, 0, 0,
                                  None)
    assert rc == -1
    assert b"null ctx" in lib.stencil_last_error()
    assert lib.stencil_version().startswith(b"b300-stencil")


def test_header_compiles_as_c_and_links(lib, tmp_path):
    """include/stencil.h is plain C: a C99 program that takes the address of
    every declared entry point compiles with -Wall -Werror and links against
    the library (nothing is called: no GPU needed)."""
    import subprocess
    names = sorted(declared_symbols())
    src = tmp_path / "use_abi.c"
    body = "\n".join(f"  fns[{i}] = (void (*)(void)){n};" for i, n in enumerate(names))
    src.write_text('#include "stencil.h"\n#include <stddef.h>\n'
                   f"void (*fns[{len(names)}])(void);\n"
                   "int main(void) {\n" + body + "\n  return fns[0] == NULL;\n}\n")
    libdir = os.path.dirname(lib._name)
    res = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-Wno-pedantic", "-I",
                          os.path.join(ROOT, "include"), str(src), "-o", str(tmp_path / "use_abi"),
                          "-L", libdir, "-lstencil", f"-Wl,-rpath,{libdir}"],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
