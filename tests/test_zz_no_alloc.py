"""The no-allocation entry point against the regular one and against the oracle.

rad_spectrum_noalloc exists for callers that cannot let the library allocate device memory
(for example when another framework's caching allocator already holds the GPU's memory,
or inside a loop where cudaMalloc/cudaFree would synchronize the device). It keeps its
scratch in one fixed 32 MiB device array inside the library. These checks call it
through the C ABI twice in a row (the second call reuses the array the first one left
behind), on the legacy default stream and on a stream of the caller's own, and compare
each result with rad_spectrum's and with the FP64 oracle's, under the mixed-precision
tolerance used by the other GPU tests. They also check that a call leaves the device's free
memory unchanged, and that a device-side data error comes back as RAD_EDATA with the cube
untouched and does not disturb the next call. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import paper_1910_10391_gb300 as rad
from paper_1910_10391_gb300 import inputs as I

from helpers import MODE_ORC, assert_mixed_close

pytestmark = pytest.mark.gpu


def _cases():
    ens = (I.channeling(8, 10e9, +1, 2000, 5e-9, seed=2), I._ensemble_grid(10e9, 20.0, 64, 16))
    L = I.lognormal_lengths(24, seed=4, median=1000, lo=200, hi=5000)
    batch = (I.channeling(24, 20e9, -1, L, 5e-9, seed=4), I._ensemble_grid(20e9, 20.0, 37, 5))
    return [("ensemble", ens, rad.RAD_CLASSICAL), ("lognormal", batch, rad.RAD_SPIN_HALF),
            ("undulator", I.workload_undulator_4096(), rad.RAD_CLASSICAL)]


@pytest.mark.parametrize("own_stream", [False, True], ids=["default-stream", "own-stream"])
@pytest.mark.parametrize("name,case,mode", _cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_noalloc_matches_regular_entry_twice(name, case, mode, own_stream):
    import torch
    tr, grid = case
    inp = rad.DeviceInputs(tr, grid)
    n = inp.n_omega * inp.n_angles
    ref = torch.empty(n, dtype=torch.float64, device="cuda")
    rc = rad.rad_spectrum(*inp.args(), mode, rad.RAD_MIXED, ref, None, None, 0, None, 0)
    assert rc == rad.RAD_OK, rad.rad_status_string(rc)
    torch.cuda.synchronize()
    assert rad.rad_device_status(1) == rad.RAD_OK
    ref_np = ref.view(inp.n_omega, inp.n_angles).cpu().numpy()
    orc = O.spectrum_cube(tr, grid, MODE_ORC[mode])
    stream = torch.cuda.Stream() if own_stream else None
    outs = [torch.full((n,), np.nan, dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    for k, out in enumerate(outs):
        free0 = torch.cuda.mem_get_info()[0]
        rc = rad.rad_spectrum_noalloc(inp.samples, inp.offsets, inp.gamma, inp.energy, inp.weight, inp.hw,
                                      inp.tx, inp.ty, mode, out, stream)
        assert rc == rad.RAD_OK, rad.rad_status_string(rc)
        if k == 1:  # the first call may load the library's device code; the second finds it loaded
            assert torch.cuda.mem_get_info()[0] == free0
        got = out.view(inp.n_omega, inp.n_angles).cpu().numpy()
        assert np.all(np.isfinite(got))
        assert_mixed_close(got, ref_np)
        assert_mixed_close(got, orc)


def test_noalloc_data_error_leaves_the_cube_untouched():
    """A non-finite sample is caught on the device: RAD_EDATA, the cube keeps what it held, and
    the next call (which clears the shared control words) computes normally."""
    import torch
    tr, grid = _cases()[0][1]
    good = rad.DeviceInputs(tr, grid)
    bad_tr = I.Trajectories(tr.samples.copy(), tr.offsets, tr.gamma, tr.energy_eV, tr.weight)
    bad_tr.samples[tr.offsets[3] + 17, 1] = np.nan
    bad = rad.DeviceInputs(bad_tr, grid)
    n = good.n_omega * good.n_angles
    out = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rc = rad.rad_spectrum_noalloc(bad.samples, bad.offsets, bad.gamma, bad.energy, bad.weight, bad.hw,
                                  bad.tx, bad.ty, rad.RAD_CLASSICAL, out)
    assert rc == rad.RAD_EDATA, rad.rad_status_string(rc)
    assert torch.all(out == 7.0)
    rc = rad.rad_spectrum_noalloc(good.samples, good.offsets, good.gamma, good.energy, good.weight, good.hw,
                                  good.tx, good.ty, rad.RAD_CLASSICAL, out)
    assert rc == rad.RAD_OK, rad.rad_status_string(rc)
    got = out.view(good.n_omega, good.n_angles).cpu().numpy()
    assert_mixed_close(got, O.spectrum_cube(tr, grid, O.CLASSICAL))


def test_noalloc_rejects_oversize_requests():
    import torch
    tr, grid = _cases()[0][1]
    inp = rad.DeviceInputs(tr, grid)
    out = torch.empty(16, dtype=torch.float64, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    # 2048 energies x 4096 directions = 8.4M bins > 4,194,272: rejected before any device work
    rc = rad.load().rad_spectrum_noalloc(p(inp.samples), inp.n_samples, p(inp.offsets), inp.n_particles,
                                         p(inp.gamma), p(inp.energy), None, p(inp.hw), 2048, p(inp.tx),
                                         p(inp.ty), 4096, 0, p(out), None)
    assert rc == rad.RAD_ETOOBIG
    assert "32 MiB" in rad.rad_status_string(rc)
