"""The C-ABI library loads and exports every entry point include/rad.h declares.

No compute call runs here (there is no GPU in this suite); only host-side argument
checks that return before any CUDA work is enqueued.
"""
import ctypes

import pytest

import paper_1910_10391_gb300 as rad


@pytest.fixture(scope="module")
def lib():
    return rad.load()


def test_exports_every_declared_symbol(lib):
    names = rad.header_symbols()
    assert "rad_spectrum" in names and "rad_plan_create" in names and len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for code in range(7):
        s = rad.rad_status_string(code)
        assert isinstance(s, str) and s
    assert "sm_103a" in rad.rad_version()


def test_invalid_shapes_rejected_before_device_work(lib):
    h = ctypes.c_void_p()
    assert lib.rad_plan_create(-1, 0, 1, 1, 0, 0, 1, 0, ctypes.byref(h)) == rad.RAD_EINVAL
    assert lib.rad_plan_create(0, 0, 1, 1, 7, 0, 1, 0, ctypes.byref(h)) == rad.RAD_EINVAL   # mode
    assert lib.rad_plan_create(0, 0, 1, 1, 0, 9, 1, 0, ctypes.byref(h)) == rad.RAD_EINVAL   # precision
    assert lib.rad_plan_create(0, 0, 1, 1, 0, 0, 4, 0, ctypes.byref(h)) == rad.RAD_EINVAL   # bins need n_bins
    assert lib.rad_plan_create(3, 2, 1, 1, 0, 0, 1, 0, ctypes.byref(h)) == rad.RAD_EINVAL   # < 2 samples each
    assert lib.rad_plan_create(0, 0, 1, 1, 0, 0, 1, 0, None) == rad.RAD_EINVAL
    assert lib.rad_plan_execute(None, *([None] * 13), 0, None) == rad.RAD_EINVAL
    assert lib.rad_graph_launch(None, None) == rad.RAD_EINVAL
    assert lib.rad_plan_set_shape(None, 2, 8, 64, 1) == rad.RAD_EINVAL
    rc = lib.rad_spectrum(None, 0, None, 0, None, None, None, None, 1, None, None, None, 1, 5, 0,
                          None, None, None, 0, None, 0, None)
    assert rc == rad.RAD_EINVAL
