"""Uneven-length batches through one persistent, graph-captured launch with an autotuned shape.

256 electrons of the 20 GeV lognormal-length generator (lengths 2k..200k samples, median 20k)
on the full 1024-energy x 32x32-direction grid, spin-1/2: the graph replay is compared with
the FP64 oracle on 64 seeded bins (every bin over all 256 particles).
"""
import numpy as np
import pytest

import oracle as O
import paper_1910_10391_gb300 as rad
from paper_1910_10391_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_lognormal_batch_graph_autotuned():
    import torch
    tr, grid = I.workload_electron_batch(n_particles=4096, particles=np.arange(256))
    tr.weight[:] = 1.0
    inp = rad.DeviceInputs(tr, grid)
    plan = rad.Plan(inp.n_samples, inp.n_particles, inp.n_omega, inp.n_angles, rad.RAD_SPIN_HALF,
                    rad.RAD_MIXED, 1, 0)
    # tune on a 16-particle slice, then apply the shape to the full plan
    sub = tr.subset(range(16))
    si = rad.DeviceInputs(sub, grid)
    tp = rad.Plan(si.n_samples, 16, si.n_omega, si.n_angles, rad.RAD_SPIN_HALF, rad.RAD_MIXED, 1, 0)
    tmp = torch.empty(si.n_omega * si.n_angles, dtype=torch.float64, device="cuda")
    assert tp.autotune(*si.args(), tmp, None, None, None, budget_ms=20000) == 0
    d = dict(kv.split("=") for kv in tp.describe().split())
    assert plan.set_shape(int(d["R"]), int(d["NW"]), int(d["T"]), 1) == 0
    tp.close()
    out = torch.zeros(inp.n_omega * inp.n_angles, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = plan.graph(*inp.args(), out, None, None, None, stream=s)
        assert g.launch(s) == 0
    s.synchronize()
    assert rad.rad_device_status(1) == rad.RAD_OK
    cube = out.view(inp.n_omega, inp.n_angles).cpu().numpy()
    rng = np.random.default_rng(7)
    bi = rng.integers(0, inp.n_omega, 64)
    bj = rng.integers(0, inp.n_angles, 64)
    ref = O.spectrum_bins(tr, grid, O.SPIN_HALF, bi, bj)
    got = cube[bi, bj]
    peak = cube.max()
    sel = ref >= 1e-3 * peak
    assert sel.sum() >= 16
    rel = np.abs(got[sel] - ref[sel]) / ref[sel]
    assert rel.max() <= 1e-4, rel.max()
    assert np.all(np.abs(got - ref)[~sel] <= 1e-7 * peak)
    g.close()
    plan.close()
