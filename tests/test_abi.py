"""C-ABI checks that need no GPU: the library builds, loads, exports every symbol the
header declares, and rejects invalid arguments before touching the device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "flbm.h")


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__ as ge

    return ge._cuda_build_module().build()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(flbm_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("flbm_create", "flbm_create_ex", "flbm_step", "flbm_stats", "flbm_destroy",
                     "flbm_init_uniform", "flbm_get_populations", "flbm_set_populations",
                     "flbm_save", "flbm_load", "flbm_last_error", "flbm_batch_create",
                     "flbm_batch_step", "flbm_batch_stats"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in _declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for n in _declared_functions():
        assert hasattr(lib, n)


def test_python_binding_has_the_same_names(lib_path):
    import paper_2602_16486_gb300.flbm as fb

    for n in _declared_functions():
        assert callable(getattr(fb, n)), n


def test_argument_validation_without_gpu(lib_path):
    import paper_2602_16486_gb300 as fl

    lam27 = np.full(27, 1.2)
    lam9 = np.full(9, 1.2)
    cases = [
        (fl.FLBM_D2Q9, (8, 8, 2), lam9, 1e-4, 1.0, "nz"),
        (7, (8, 8, 1), lam9, 1e-4, 1.0, "lattice"),
        (fl.FLBM_D3Q27, (0, 8, 8), lam27, 1e-4, 1.0, "dims"),
        (fl.FLBM_D3Q27, (8, 70000, 8), lam27, 1e-4, 1.0, "65535"),
        (fl.FLBM_D3Q27, (65536, 65535, 2), lam27, 1e-4, 1.0, "2^32"),
        (fl.FLBM_D3Q27, (8, 8, 8), lam27, -1.0, 1.0, "kBT"),
        (fl.FLBM_D3Q27, (8, 8, 8), lam27, 1e-4, 0.0, "rho0"),
        (fl.FLBM_D3Q27, (8, 8, 8), np.r_[lam27[:10], 2.5, lam27[11:]], 1e-4, 1.0, "lambda[10]"),
        (fl.FLBM_D3Q27, (8, 8, 8), np.r_[lam27[:10], 0.0, lam27[11:]], 1e-4, 1.0, "lambda[10]"),
        (fl.FLBM_D2Q9, (8, 8, 1), np.r_[lam9[:4], np.nan, lam9[5:]], 1e-4, 1.0, "lambda[4]"),
    ]
    for lattice, dims, lam, kBT, rho0, word in cases:
        with pytest.raises(fl.FlbmError) as ei:
            fl.flbm_create(lattice, dims, lam, kBT, rho0, 0)
        assert ei.value.status == fl.FLBM_EINVAL
        assert word in str(ei.value)
    with pytest.raises(fl.FlbmError) as ei:
        fl.flbm_create_ex(fl.FLBM_D3Q27, (8, 8, 8), lam27, 1e-4, 1.0, 0, storage=5)
    assert ei.value.status == fl.FLBM_EINVAL
    with pytest.raises(ValueError):
        fl.flbm_create(fl.FLBM_D3Q27, (8, 8, 8), lam9, 1e-4, 1.0, 0)


def test_required_bytes_and_null_handles(lib_path):
    import paper_2602_16486_gb300 as fl

    assert fl.flbm_required_bytes(fl.FLBM_D3Q27, (256, 256, 256), fl.FLBM_FP32) == 27 * 256 ** 3 * 4
    assert fl.flbm_required_bytes(fl.FLBM_D3Q27, (256, 256, 256), fl.FLBM_BF16) == 27 * 256 ** 3 * 2
    assert fl.flbm_required_bytes(fl.FLBM_D2Q9, (64, 64, 1), fl.FLBM_FP16) == 9 * 64 * 64 * 2
    assert fl.flbm_required_bytes(fl.FLBM_D2Q9, (64, 64, 2), fl.FLBM_FP32) == 0
    lib = ctypes.CDLL(lib_path)
    lib.flbm_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    assert lib.flbm_step(None, 1) == fl.FLBM_EINVAL
    lib.flbm_get_step.restype = ctypes.c_int64
    lib.flbm_get_step.argtypes = [ctypes.c_void_p]
    assert lib.flbm_get_step(None) == -1
    lib.flbm_destroy.argtypes = [ctypes.c_void_p]
    lib.flbm_destroy(None)  # no-op
    lib.flbm_last_error.restype = ctypes.c_char_p
    assert lib.flbm_last_error()


def test_package_refuses_to_import_without_library(tmp_path):
    # The binding has no fallback: a missing library is an ImportError.
    code = (
        "import sys, importlib.util, os\n"
        f"spec = importlib.util.spec_from_file_location('fb', r'{ROOT}/paper_2602_16486_gb300/flbm.py')\n"
        "m = importlib.util.module_from_spec(spec)\n"
        "import builtins\n"
        "orig = os.path.exists\n"
        "os.path.exists = lambda p: False if p.endswith('libflbm.so') else orig(p)\n"
        "try:\n"
        "    spec.loader.exec_module(m)\n"
        "except ImportError as e:\n"
        "    print('IMPORT-ERROR', e)\n"
    )
    res = subprocess.run(["python", "-c", code], capture_output=True, text=True)
    assert "IMPORT-ERROR" in res.stdout
