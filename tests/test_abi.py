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
    assert L.lu_factor(4, ctypes.c_void_p(16), 4, ctypes.c_void_p(16), -1) == -5
    assert L.lu_factor(4, ctypes.c_void_p(16), 4, ctypes.c_void_p(16), 1025) == -5
    assert L.lu_solve(-2, 1, None, None, None) == -1
    assert L.lu_factor_ex(None, 0, 4, None, 4, None, None, None) == _lib.LU_ERR_HANDLE
    assert L.lu_potrf_ex(None, 0, 4, None, 4, None, None) == _lib.LU_ERR_HANDLE
    o = pkg.LuOpts()
    L.lu_default_opts(ctypes.byref(o))
    assert (o.nb, o.lookahead, o.steal) == (256, 1, 1)
    assert L.lu_launch_count() >= 0
    assert L.lu_peak_fma(0, 0, 256, 1, ctypes.c_void_p(16), None) == -2
    assert L.lu_peak_fma(0, 1, 100, 1, ctypes.c_void_p(16), None) == -3
    assert L.lu_peak_fma(1, 1, 256, 1, None, None) == -5
    assert L.lu_peak_fma_chains() == 16


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "lu_gb300.h"\nint main(void){lu_opts o; lu_default_opts(&o); return o.nb == 256 ? 0 : 1;}\n')
    inc = os.path.join(os.path.dirname(_lib.HEADER))
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-c", str(src), "-I", inc, "-o", str(tmp_path / "t.o")],
                   check=True)


def test_tune_table_round_trip(built, tmp_path):
    """The nb table behind nb = 0 (lu_tune_*): set/get by (device, kind,
    ceil(log2 n)), replacement, save/load round trip, rejection of malformed
    files without partial merges, and argument checks, all on the host."""
    L = pkg.lib()
    dev = b"Test GPU"
    assert L.lu_tune_clear() == 0
    assert L.lu_tune_get(dev, pkg.LU_TU_BF16X6, 16384) == 0
    assert L.lu_tune_set(dev, pkg.LU_TU_BF16X6, 16384, 512, 80.5) == 0
    # one bucket per power of two: (8192, 16384] shares the entry, 16385 does not
    assert L.lu_tune_get(dev, pkg.LU_TU_BF16X6, 8193) == 512
    assert L.lu_tune_get(dev, pkg.LU_TU_BF16X6, 16385) == 0
    assert L.lu_tune_get(dev, pkg.LU_TU_BF16, 16384) == 0
    assert L.lu_tune_get(b"Other GPU", pkg.LU_TU_BF16X6, 16384) == 0
    assert L.lu_tune_set(dev, pkg.LU_TU_BF16X6, 12000, 384, 70.0) == 0  # same key: replaced
    assert L.lu_tune_get(dev, pkg.LU_TU_BF16X6, 16384) == 384
    assert L.lu_tune_set(dev, pkg.LU_TUNE_F64, 8192, 256, 300.0) == 0
    assert L.lu_tune_set(dev, pkg.LU_TU_FP8, 32768, 128, 200.0) == 0
    # argument checks
    assert L.lu_tune_set(b"", pkg.LU_TUNE_F64, 8192, 256, 0.0) == -1
    assert L.lu_tune_set(b"a\tb", pkg.LU_TUNE_F64, 8192, 256, 0.0) == -1
    assert L.lu_tune_set(dev, pkg.LU_FULL_F64, 8192, 256, 0.0) == -2
    assert L.lu_tune_set(dev, 7, 8192, 256, 0.0) == -2
    assert L.lu_tune_set(dev, pkg.LU_TUNE_F64, 0, 256, 0.0) == -3
    assert L.lu_tune_set(dev, pkg.LU_TUNE_F64, 8192, 0, 0.0) == -4
    assert L.lu_tune_set(dev, pkg.LU_TUNE_F64, 8192, 1025, 0.0) == -4
    assert L.lu_tune_set(dev, pkg.LU_TU_FP8, 8192, 192, 0.0) == -4
    assert L.lu_tune_save(None) == -1 and L.lu_tune_load(None) == -1
    path = tmp_path / "tune.txt"
    assert L.lu_tune_save(str(path).encode()) == 0
    lines = path.read_text().splitlines()
    assert sorted(lines) == sorted(["Test GPU\t6\t14\t384\t70", "Test GPU\t100\t13\t256\t300",
                                    "Test GPU\t2\t15\t128\t200"])
    assert L.lu_tune_clear() == 0 and L.lu_tune_get(dev, pkg.LU_TU_BF16X6, 16384) == 0
    assert L.lu_tune_load(str(path).encode()) == 0
    assert L.lu_tune_get(dev, pkg.LU_TU_BF16X6, 16384) == 384
    assert L.lu_tune_get(dev, pkg.LU_TUNE_F64, 5000) == 256
    assert L.lu_tune_get(dev, pkg.LU_TU_FP8, 20000) == 128
    # malformed files are rejected whole
    for bad in ["Test GPU\t6\t14\n", "Test GPU\t6\t14\t384\t70\textra\n", "\t6\t14\t384\t70\n",
                "Test GPU\t9\t14\t384\t70\n", "Test GPU\t2\t14\t192\t70\n", "Test GPU\t6\t99\t384\t70\n"]:
        f = tmp_path / "bad.txt"
        f.write_text("New GPU\t6\t14\t512\t1\n" + bad)
        assert L.lu_tune_load(str(f).encode()) == pkg.LU_ERR_IO, bad
        assert L.lu_tune_get(b"New GPU", pkg.LU_TU_BF16X6, 16384) == 0
    assert L.lu_tune_load(str(tmp_path / "missing.txt").encode()) == pkg.LU_ERR_IO
    assert L.lu_tune_nb(None, pkg.LU_TUNE_F64, 64, None, 0, 1, None, None, None) == _lib.LU_ERR_HANDLE
    assert L.lu_tune_clear() == 0


def test_tune_plan_table_round_trip(built, tmp_path):
    """Tuned plans (lu_tune_plan_set/get): nb with a per-step schedule, the
    right update's SM reserve and the look-ahead depth survive a save/load
    round trip; a plain nb entry keeps the short line format; malformed plans
    are rejected whole."""
    import ctypes as C
    L = pkg.lib()
    dev = b"Plan GPU"
    assert L.lu_tune_clear() == 0
    sched = (C.c_int32 * 4)(512, 384, 256, 128)
    assert L.lu_tune_plan_set(dev, pkg.LU_TU_BF16X6, 16384, 256, 25, 2, sched, 4, 24, 75.0) == 0
    assert L.lu_tune_set(dev, pkg.LU_TUNE_F64, 8192, 128, 300.0) == 0
    nb, res, dep, cnt, pf = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
    out = (C.c_int32 * 8)()
    assert L.lu_tune_plan_get(dev, pkg.LU_TU_BF16X6, 10000, C.byref(nb), C.byref(res), C.byref(dep), out, 8,
                              C.byref(cnt), C.byref(pf)) == 1
    assert (nb.value, res.value, dep.value, cnt.value, pf.value) == (256, 25, 2, 4, 24)
    assert list(out[:4]) == [512, 384, 256, 128]
    assert L.lu_tune_get(dev, pkg.LU_TU_BF16X6, 16384) == 256
    assert L.lu_tune_plan_get(dev, pkg.LU_TU_BF16, 16384, None, None, None, None, 0, None, None) == 0
    # argument checks
    assert L.lu_tune_plan_set(dev, pkg.LU_TU_FP8, 16384, 128, 0, 1, (C.c_int32 * 1)(192), 1, 0, 0.0) == -7
    assert L.lu_tune_plan_set(dev, pkg.LU_TU_BF16, 16384, 256, -1, 1, None, 0, 0, 0.0) == -5
    assert L.lu_tune_plan_set(dev, pkg.LU_TU_BF16, 16384, 256, 0, 3, None, 0, 0, 0.0) == -6
    assert L.lu_tune_plan_set(dev, pkg.LU_TU_BF16, 16384, 256, 0, 1, None, 2, 0, 0.0) == -8
    path = tmp_path / "plan.txt"
    assert L.lu_tune_save(str(path).encode()) == 0
    lines = sorted(path.read_text().splitlines())
    assert lines == sorted(["Plan GPU\t6\t14\t256\t75\t25\t2\t512,384,256,128\t24", "Plan GPU\t100\t13\t128\t300"])
    assert L.lu_tune_clear() == 0 and L.lu_tune_load(str(path).encode()) == 0
    assert L.lu_tune_plan_get(dev, pkg.LU_TU_BF16X6, 16384, C.byref(nb), C.byref(res), C.byref(dep), out, 2,
                              C.byref(cnt), C.byref(pf)) == 1
    assert (nb.value, res.value, dep.value, cnt.value, pf.value) == (256, 25, 2, 4, 24)
    assert list(out[:2]) == [512, 384]
    # a plan without a schedule
    assert L.lu_tune_plan_set(dev, pkg.LU_TU_BF16, 4096, 192, 12, 1, None, 0, 0, 5.0) == 0
    assert L.lu_tune_save(str(path).encode()) == 0
    assert "Plan GPU\t0\t12\t192\t5\t12\t1\t-" in path.read_text().splitlines()
    for bad in ["Plan GPU\t6\t14\t256\t75\t25\t2\t512,,256\n", "Plan GPU\t6\t14\t256\t75\t25\t3\t-\n",
                "Plan GPU\t6\t14\t256\t75\t25\t2\t2000\n", "Plan GPU\t6\t14\t256\t75\t25\n",
                "Plan GPU\t2\t14\t128\t75\t0\t1\t128,192\n", "Plan GPU\t6\t14\t256\t75\t25\t2\t256x\n",
                "Plan GPU\t6\t14\t256\t75\t25\t2\t-\t-3\n", "Plan GPU\t6\t14\t256\t75\t25\t2\t-\t16\t1\n"]:
        f = tmp_path / "bad.txt"
        f.write_text("New GPU\t6\t14\t512\t1\n" + bad)
        assert L.lu_tune_load(str(f).encode()) == pkg.LU_ERR_IO, bad
    assert L.lu_tune_get(b"New GPU", pkg.LU_TU_BF16X6, 16384) == 0
    # a long schedule (over the 1 KiB read buffer) round-trips
    long = (C.c_int32 * 600)(*([64] * 600))
    assert L.lu_tune_plan_set(dev, pkg.LU_TU_BF16X6, 32768, 64, 0, 0, long, 600, 0, 1.0) == 0
    assert L.lu_tune_save(str(path).encode()) == 0
    assert L.lu_tune_clear() == 0 and L.lu_tune_load(str(path).encode()) == 0
    assert L.lu_tune_plan_get(dev, pkg.LU_TU_BF16X6, 32768, None, None, None, None, 0, C.byref(cnt), None) == 1
    assert cnt.value == 600
    assert L.lu_tune_clear() == 0
