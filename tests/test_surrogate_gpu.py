"""End-to-end surrogate at its 1 % contract: what the network gains over the kernel alone.

Trains a 3-model ensemble on 32768 kernel spectra (24 Lorentz factors over the whole input
domain, entry angles over the whole training domain), calibrates its error estimates on 16
validation beams, then evaluates 4 held-out beams of 512 entries (one Lorentz factor per beam,
two near each end of the range, entry angles with the ensemble workloads' divergence 0.3 theta_L)
against the kernel, with fallback until the beam mean's calibrated estimate is at most 1 %.
Checks, with no slack: each beam's mean spectrum is within its calibrated estimate of the
kernel's and that estimate is at most 1 %; the training loss falls; the surrogate's inference is
far faster than the kernel; and with the fallback included the beam means come out faster than
from the kernel alone.
"""
import numpy as np
import pytest

from paper_1910_10391_gb300 import surrogate as S

pytestmark = pytest.mark.gpu


def test_surrogate_meets_its_one_percent_contract():
    cfg = S.Config(n_gamma_train=24, n_models=3, steps=6000, batch=512, fallback_rel=0.01, calib_gamma_bins=2)
    x0, th, g = S.sample_entries(cfg, 32768, seed=5, discrete_gamma=True)
    bins = S.kernel_bins(cfg, x0, th, g)
    vx0, vth, vg, vb = S.sample_beams(cfg, 16, 48, seed=7, divergence=cfg.beam_divergence)
    sur = S.Surrogate(cfg)
    hist = sur.fit(S.raw_inputs(cfg, x0, th, g), bins, S.raw_inputs(cfg, vx0, vth, vg),
                   S.kernel_bins(cfg, vx0, vth, vg), vb)
    first = [h[2] for h in hist if h[1] == 0]
    last = [h[2] for h in hist if h[1] == cfg.steps - 1]
    assert all(l < f / 5 for f, l in zip(first, last))
    lo, hi = cfg.gamma_lo, cfg.gamma_hi
    gammas = [lo * 1.02, lo * 1.1, hi / 1.1, hi / 1.02]
    hx0, hth, hg, hb = S.sample_beams(cfg, 4, 512, seed=6, divergence=cfg.beam_divergence, gammas=gammas)
    rep = S.evaluate(sur, hx0, hth, hg, hb)
    print({k: v for k, v in rep.items() if k != "per_beam"})
    print(rep["per_beam"])
    for e in rep["per_beam"]:
        assert e["error"] <= e["estimate"] <= cfg.fallback_rel, e
    assert rep["t_predict_all_s"] * 10 < rep["t_kernel_s"]
    assert rep["gain"] > 1.0, rep["gain"]
    sur.close()
