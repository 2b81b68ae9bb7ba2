"""Failure detection on the GPU without a fault: a bounded device-side wait that runs out.

Every staging kernel waits for its bulk copies with a bounded mbarrier wait; when the limit runs
out it records RAD_ETIMEOUT and returns. rad_selftest_bounded_wait runs that wait on a barrier phase
that nothing completes: the call must end with RAD_ETIMEOUT in the status word after about the
wait's time limit, and the context must stay usable for the next computation.
"""
import time

import numpy as np
import pytest

import oracle as O
import paper_1910_10391_gb300 as rad
from paper_1910_10391_gb300 import inputs as I

from helpers import assert_mixed_close, gpu_cube

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_stays_usable():
    import torch
    assert rad.rad_device_status(1) in (rad.RAD_OK, rad.RAD_ETIMEOUT, rad.RAD_EDATA)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert rad.rad_selftest_bounded_wait(None) == rad.RAD_OK
    st = rad.rad_device_status(1)  # waits for the device
    dt = time.perf_counter() - t0
    assert st == rad.RAD_ETIMEOUT, rad.rad_status_string(st)
    assert 1.0 < dt < 30.0, dt
    assert rad.rad_device_status(1) == rad.RAD_OK  # cleared
    # the next computation runs normally
    tr, grid = I.workload_undulator_4096()
    got = gpu_cube(tr, grid, rad.RAD_CLASSICAL, rad.RAD_MIXED)["cube"]
    assert_mixed_close(got, O.spectrum_cube(tr, grid, O.CLASSICAL))
