"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/adp.h (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "adp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(adp_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2502_09758_gb300 import build
    return build.build()


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for required in ("adp_lower_solve", "adp_hypergrad", "adp_upper_loss", "adp_maid_step",
                     "adp_problem_create", "adp_problem_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_2502_09758_gb300 import adp
    assert sorted(adp.EXPORTS) == declared_functions()
    adp.load_library(lib_path)     # signatures attach without a GPU


def test_library_has_no_cpu_fallback_symbols(lib_path):
    # the product library must not link or embed the oracle
    lib = ctypes.CDLL(lib_path)
    for name in ("orc_conv", "orc_fista", "orc_maid_step"):
        assert not hasattr(lib, name)


def test_null_handles_are_rejected_before_any_device_work(lib_path):
    """Argument checks come first: a null problem gives ADP_EINVAL (and the
    queries their neutral values) without touching a device, so this runs
    on a machine without one."""
    from paper_2502_09758_gb300 import adp
    lib = adp.load_library(lib_path)
    nul = None
    assert lib.adp_apply_B_bf16(nul, nul, nul, nul) == adp.ADP_EINVAL
    assert lib.adp_apply_Bt_bf16(nul, nul, nul, nul) == adp.ADP_EINVAL
    assert lib.adp_set_fft(nul, 1) == adp.ADP_EINVAL
    assert lib.adp_set_fft(nul, 0) == adp.ADP_EINVAL
    assert lib.adp_fft_enabled(nul) == 0
    assert lib.adp_bf16_grid_size(nul) == 0
    assert lib.adp_bf16_prep_ms_last(nul) == -1.0
    assert lib.adp_apply_B(nul, nul, nul, nul) == adp.ADP_EINVAL
    assert b"null problem" in lib.adp_last_error()
