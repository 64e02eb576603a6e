"""The C ABI library builds for sm_103a, loads, exports every symbol include/hot.h declares,
and rejects invalid arguments before touching a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hot():
    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import hot as h
    return h


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hot.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hot_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(hot):
    names = declared_functions()
    assert len(names) >= 12
    lib = ctypes.CDLL(hot._LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(hot.SIGNATURES)


def test_library_targets_sm103a(hot):
    # the fatbin carries an sm_103a cubin: cuobjdump-free check through the build command
    from paper_0907_4027_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_invalid_arguments_fail_before_device_work(hot):
    lib = hot.lib
    h = ctypes.c_void_p()
    assert lib.hot_create(None, 8, 8, 1e-5, 1e-6, 1e-3, None) == hot.HOT_EINVAL
    assert lib.hot_create(ctypes.byref(h), 0, 8, 1e-5, 1e-6, 1e-3, None) == hot.HOT_EINVAL
    assert h.value is None
    assert "invalid size" in hot.hot_last_error()
    assert lib.hot_create(ctypes.byref(h), 65536, 65536, 1e-5, 1e-6, 1e-3, None) == hot.HOT_EINVAL
    assert lib.hot_create(ctypes.byref(h), 8, 8, -1.0, 1e-6, 1e-3, None) == hot.HOT_EINVAL
    assert lib.hot_create(ctypes.byref(h), 8, 8, 1e-5, float("nan"), 1e-3, None) == hot.HOT_EINVAL
    assert lib.hot_set_traps(None, 1, None, None) == hot.HOT_EINVAL
    assert lib.hot_gsw(None, 1, None, None) == hot.HOT_EINVAL
    assert lib.hot_phase_out(None, None, 0, 0) == hot.HOT_EINVAL
    assert lib.hot_get_fields(None, None, None) == hot.HOT_EINVAL
    assert lib.hot_set_precision(None, 0) == hot.HOT_EINVAL
    assert lib.hot_sync(None) == hot.HOT_EINVAL
    assert lib.hot_get_state(None, None, None) == hot.HOT_EINVAL
    assert lib.hot_set_state(None, None, None) == hot.HOT_EINVAL
    assert lib.hot_get_phasors(None, None) == hot.HOT_EINVAL
    assert lib.hot_set_phasors(None, None) == hot.HOT_EINVAL
    assert lib.hot_set_once(None, 1) == hot.HOT_EINVAL
    assert lib.hot_kernel_launches(None) == 0
    lib.hot_destroy(None)


def test_python_errors_carry_the_status(hot):
    with pytest.raises(hot.HotError) as ei:
        hot.hot_create(0, 0, 1e-5, 1e-6, 1e-3)
    assert ei.value.status == hot.HOT_EINVAL
