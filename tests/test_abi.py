"""The C-ABI library: it builds for sm_103a, loads, exports every function that
include/ccgf.h declares, and validates arguments on the host (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ccgf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ccgf_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_07478_gb300 import binding, build_lib
    if not os.path.exists(binding.LIB_PATH):
        build_lib.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ccgf_build_intermediates", "ccgf_sigma_ip", "ccgf_sigma_ea", "ccgf_solve_gf"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_export_list_matches_header():
    from paper_2208_07478_gb300 import binding
    assert sorted(binding.EXPORTS) == declared_functions()


def test_host_side_validation_without_gpu(lib):
    from paper_2208_07478_gb300 import binding as B
    o = B.default_options()
    assert o.prec == B.FP64 and o.tol == 1e-10 and o.restart_m == 30
    assert lib.ccgf_status_string(B.CCGF_ERR_NAN) == b"non-finite input"
    h = ctypes.c_void_p()
    assert lib.ccgf_build_intermediates(None, None, None, ctypes.byref(h)) == B.CCGF_ERR_INVALID_ARG
    s = B.System()
    s.kmesh[:] = [0, 1, 1]
    assert lib.ccgf_build_intermediates(ctypes.byref(s), None, None, ctypes.byref(h)) == B.CCGF_ERR_INVALID_ARG
    assert b"kmesh" in lib.ccgf_last_error()
    assert lib.ccgf_sigma_ip(None, 0, 1, None, None, 0, None) == B.CCGF_ERR_INVALID_ARG
    assert lib.ccgf_sigma_ip_noalloc(None, 0, 1, None, None, None) == B.CCGF_ERR_INVALID_ARG
    assert lib.ccgf_solve_gf(None, 3, 1, None, 0.01, None, None, 0, None, None) == B.CCGF_ERR_INVALID_ARG
    assert lib.ccgf_launch_count(None) == 0


def test_product_path_refuses_to_run_without_the_library(tmp_path):
    from paper_2208_07478_gb300 import binding
    with pytest.raises(FileNotFoundError):
        binding.load(str(tmp_path / "libccgf.so"))


def test_wait_bound_option_is_validated(lib):
    from paper_2208_07478_gb300 import binding as B
    h = ctypes.c_void_p()
    s = B.System()
    s.kmesh[:] = [1, 1, 1]
    for bad in (0.0, -1.0, 6.0e4 + 1.0):
        o = B.default_options(device_wait_timeout_ms=bad)
        assert lib.ccgf_build_intermediates(ctypes.byref(s), ctypes.byref(o), None, ctypes.byref(h)) == B.CCGF_ERR_INVALID_ARG
        assert b"device_wait_timeout_ms" in lib.ccgf_last_error()
    assert B.default_options().device_wait_timeout_ms == 1000.0
