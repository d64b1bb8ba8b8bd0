"""The C-ABI library builds for sm_103a and exports every entry point that
include/lcqmc.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "lcqmc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(lcqmc_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_core_api():
    names = declared_functions()
    for n in ("lcqmc_create", "lcqmc_update", "lcqmc_measure", "lcqmc_submit", "lcqmc_poll",
              "lcqmc_destroy", "lcqmc_last_error"):
        assert n in names


def test_header_compiles_as_c(tmp_path):
    # The boundary is a C ABI: the header must compile as plain C11.
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "use.c"
    src.write_text(
        '#include "lcqmc.h"\n'
        "int use(void) {\n"
        "  lcqmc_handle h = 0; lcqmc_obs o; lcqmc_record r; lcqmc_sw_t sw = 0; lcqmc_tuning t;\n"
        "  int64_t n = 0; (void)o; (void)r; (void)t;\n"
        "  if (lcqmc_create(64, 0.5, 1.0, 8.0, 1, &h) != LCQMC_OK) return 1;\n"
        "  lcqmc_update(h, 1); lcqmc_get_records(h, &r, 1, &n); lcqmc_destroy(h);\n"
        "  lcqmc_sw_create(64, 0.44, 1, 0, &sw); lcqmc_sw_destroy(sw);\n"
        "  return (int)n;\n"
        "}\n")
    import subprocess
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-c", str(src), "-o", str(tmp_path / "use.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.fixture(scope="module")
def built_lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1810_07485_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built_lib):
    so = ctypes.CDLL(built_lib)
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_last_error_callable_without_gpu(built_lib):
    so = ctypes.CDLL(built_lib)
    so.lcqmc_last_error.restype = ctypes.c_char_p
    assert isinstance(so.lcqmc_last_error(), bytes)


def test_invalid_arguments_rejected_on_host(built_lib):
    # Argument validation happens before any CUDA call.
    from paper_1810_07485_gb300 import lcqmc
    L = lcqmc.lib()
    h = ctypes.c_void_p()
    for args in [(3, 0.5, 1.0, 1.0), (0, 0.5, 1.0, 1.0), (8, 0.75, 1.0, 1.0), (8, 0.5, -1.0, 1.0),
                 (8, 0.5, 1.0, 0.0), (8, 2.5, 1.0, 1.0), (8, 3.0, 1.0, 1.0)]:
        rc = L.lcqmc_create(args[0], args[1], args[2], args[3], 1, ctypes.byref(h))
        assert rc == -1, args


def test_sw_invalid_arguments_rejected_on_host(built_lib):
    # The Swendsen-Wang handle validates L and K before any CUDA call.
    from paper_1810_07485_gb300 import lcqmc
    L = lcqmc.lib()
    h = ctypes.c_void_p()
    for Lx, K in [(1, 0.4), (0, 0.4), (46341, 0.4), (8, -1.0), (8, float("nan")), (8, float("inf"))]:
        assert L.lcqmc_sw_create(Lx, K, 1, None, ctypes.byref(h)) == -1, (Lx, K)
        assert h.value is None
    assert L.lcqmc_sw_update(None, 1) == -1
    assert L.lcqmc_sw_sync(None) == -1
    assert b"null handle" in L.lcqmc_last_error()


@pytest.mark.parametrize("which", [0, 1])
def test_integer_rounding_forms_match_libm(built_lib, which):
    # The kernels evaluate fma(t_end - t0, u, t0) and rint(x 2^F) with integer
    # arithmetic; the same code, run on the host, must agree bit for bit with
    # the C library on a million random inputs.
    so = ctypes.CDLL(built_lib)
    bad = ctypes.c_int64(-1)
    rc = so.lcqmc_selftest(ctypes.c_int(which), ctypes.c_int64(1_000_000), ctypes.c_uint64(12345),
                           ctypes.byref(bad))
    assert rc == 0 and bad.value == 0
