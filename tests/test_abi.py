"""CPU checks of the C ABI: the library builds, loads, and exports every
function include/fbp.h declares (no compute calls: there may be no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2109_02174_gb300 import build
    build.build()
    import paper_2109_02174_gb300 as fbp
    return fbp.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fbp_plan", "fbp_plan_destroy", "fbp_workspace_bytes", "fbp_plan_query",
                     "fbp_filter", "fbp_backproject", "fbp_reconstruct", "radon_forward",
                     "fbp_last_error", "fbp_device_status", "fbp_options_default"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_options_default_and_null_checks(lib):
    import paper_2109_02174_gb300 as fbp
    o = fbp.fbp_options_default()
    assert (o.dtype, o.q_storage, o.accumulate, o.filter_path, o.i0) == (0, 0, 0, 0, 0.0)
    assert lib.fbp_options_default(None) == fbp.FBP_ERR_INVALID_ARG
    assert "NULL" in fbp.fbp_last_error()
    assert lib.fbp_plan(None, 8, 8, 8, None, 1.0, 0, None) == fbp.FBP_ERR_INVALID_ARG
    assert lib.fbp_plan_destroy(None) == fbp.FBP_OK
    assert lib.fbp_workspace_bytes(None, None) == fbp.FBP_ERR_INVALID_ARG
    assert lib.fbp_backproject(None, None, None, None) == fbp.FBP_ERR_INVALID_ARG


def test_plan_argument_errors_are_host_side(lib):
    """Bad sizes and spacings are rejected before any device work."""
    import paper_2109_02174_gb300 as fbp
    h = ctypes.c_void_p()
    for args in ((0, 10, 10, 1.0, 0), (10, 0, 10, 1.0, 0), (10, 10, 0, 1.0, 0),
                 (10, 10, 10, 0.0, 0), (10, 10, 10, -1.0, 0), (10, 10, 10, float("nan"), 0),
                 (10, 10, 10, 1.0, 9), (20000, 10, 10, 1.0, 0)):
        n, a, d, tau, flt = args
        st = lib.fbp_plan(ctypes.byref(h), n, a, d, None, tau, flt, None)
        assert st == fbp.FBP_ERR_INVALID_ARG, args
        assert h.value is None


def test_autotune_argument_errors_need_no_gpu(lib):
    import paper_2109_02174_gb300 as fbp
    t = fbp.fbp_tuning()
    assert lib.fbp_autotune(64, 90, 92, 1.0, 0, None, 0, ctypes.byref(t)) == fbp.FBP_ERR_INVALID_ARG
    assert lib.fbp_autotune(64, 90, 92, 1.0, 0, None, 4, None) == fbp.FBP_ERR_INVALID_ARG


def test_wait_settings_argument_errors_need_no_gpu(lib):
    """The wait-limit and test-hook calls check their arguments before they
    look for a device."""
    import paper_2109_02174_gb300 as fbp
    for bad in (-1.0, float("nan"), float("inf"), 1e-9, 1e5):
        assert lib.fbp_set_wait_limit(bad) == fbp.FBP_ERR_INVALID_ARG, bad
    assert "fbp_set_wait_limit" in fbp.fbp_last_error()
    assert lib.fbp_test_withhold_arrival(9, 0) == fbp.FBP_ERR_INVALID_ARG
    assert lib.fbp_test_withhold_arrival(fbp.FBP_TEST_WITHHOLD_FILTER_TC, -1) == \
        fbp.FBP_ERR_INVALID_ARG
