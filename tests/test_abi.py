"""CPU-side checks of the C ABI: the library builds, loads, and exports every
function that include/lu_gb300.h declares; argument validation answers
without touching a GPU."""
import ctypes
import os
import subprocess

import pytest

import paper_1804_07017_gb300 as pkg
from paper_1804_07017_gb300 import _lib
from paper_1804_07017_gb300 import build as libbuild


@pytest.fixture(scope="module")
def built():
    return libbuild.build()


def test_library_exports_header_symbols(built):
    declared = _lib.declared_symbols()
    assert "lu_factor" in declared and "lu_solve" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    L = pkg.lib()
    for s in declared:
        assert hasattr(L, s)
    # every declared symbol has a ctypes signature in the binding
    assert set(declared) <= set(_lib.signatures())


def test_argument_validation_without_gpu(built):
    L = pkg.lib()
    assert L.lu_factor(-1, None, 1, None, 64) == -1
    assert L.lu_factor(4, None, 4, None, 64) == -2
    assert L.lu_factor(4, ctypes.c_void_p(16), 3, ctypes.c_void_p(16), 64) == -3
    assert L.lu_factor(4, ctypes.c_void_p(16), 4, ctypes.c_void_p(16), 0) == -5
    assert L.lu_solve(-2, 1, None, None, None) == -1
    assert L.lu_factor_ex(None, 0, 4, None, 4, None, None, None) == _lib.LU_ERR_HANDLE
    o = pkg.LuOpts()
    L.lu_default_opts(ctypes.byref(o))
    assert (o.nb, o.lookahead, o.steal) == (256, 1, 1)
    assert L.lu_launch_count() >= 0


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "lu_gb300.h"\nint main(void){lu_opts o; lu_default_opts(&o); return o.nb == 256 ? 0 : 1;}\n')
    inc = os.path.join(os.path.dirname(_lib.HEADER))
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-c", str(src), "-I", inc, "-o", str(tmp_path / "t.o")],
                   check=True)
