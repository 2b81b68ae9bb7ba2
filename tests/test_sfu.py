"""Accuracy of the SFU sin/cos the mixed kernel uses on unreduced arguments.

The mixed kernel passes phase offsets of up to ~1e3 rad straight to the special-function
unit (the __sincosf intrinsic), which reduces the argument itself. This test measures the
absolute error against FP64 sin/cos over |x| up to 2e4 rad and checks the bound the error
budget uses: |err| <= 1e-6 + 2.5e-7 |x| (observed ~4e-7 near 0 and ~1.6-2.0e-7 |x| beyond).
"""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def sfu_lib():
    out = os.path.join(tempfile.mkdtemp(), "sfu_probe.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared",
                           "-Xcompiler", "-fPIC", os.path.join(HERE, "sfu_probe.cu"), "-o", out])
    return ctypes.CDLL(out)


@pytest.mark.parametrize("lo,hi", [(0.0, np.pi), (np.pi, 100 * np.pi), (100 * np.pi, 1000.0),
                                   (1000.0, 3000.0), (3000.0, 20000.0)])
def test_sfu_sincos_error_bound(sfu_lib, lo, hi):
    rng = np.random.default_rng(int(lo) + 1)
    n = 1 << 20
    x = (rng.uniform(lo, hi, n) * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    s = np.empty_like(x)
    c = np.empty_like(x)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert sfu_lib.sfu_eval(p(x), p(s), p(c), n) == 0
    xd = x.astype(np.float64)
    err = np.maximum(np.abs(s - np.sin(xd)), np.abs(c - np.cos(xd)))
    assert np.all(err <= 1e-6 + 2.5e-7 * np.abs(xd))
