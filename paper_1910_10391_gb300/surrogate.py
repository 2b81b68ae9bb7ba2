"""Learned surrogate for per-particle planar-channeling spectra, with the exact kernel as fallback.

Entry conditions (x0/d_p, theta0/theta_L, gamma) of a positron in the harmonic planar well
(no multiple scattering, 100 um, 8192 samples) map to log10 of its spectrum dI/d(hw) in 8
radial bins of the emission angle, at 256 photon energies hw/E log-spaced in [1e-4, 0.5]
(BCK spin-1/2 model). Training spectra come from rad_spectrum_particles; the network (3 ->
256 -> 256 -> 256 -> 2048, GELU) is trained with the library's own BF16 tensor-core kernels.
An ensemble of networks gives an error estimate per entry; entries whose estimate exceeds
`fallback_rel` are recomputed with the exact kernel.

Angle grid per gamma: 32 x 32 cells over +-(theta_L + 3/gamma); radial bins of |theta| in
[0, theta_L + 3/gamma). Motion without scattering stays in the x-z plane, so the spectrum is
symmetric in theta_y: only the theta_y > 0 half is computed, with doubled cell solid angles.

Frequency alignment: the spectra are sharp harmonic lines whose positions move with the
transverse energy and gamma. The fundamental of the transverse motion has a closed form in the
harmonic well (channeled: 2 theta_L/d_p; over the barrier: 2 pi theta_L/(d_p arcsin(eps^-1/2))),
which with the mean squared transverse velocity gives the first line hw1 = 2 gamma^2 hbar c
Omega / (1 + gamma^2 <v^2>). Because the photon-energy grid is log-uniform, shifting an entry's
labels by the whole number of grid steps that puts hw1 at a fixed index is exact; the network
predicts on that extended, aligned grid (masked loss outside each entry's window) and sees
the remaining fraction of a step as an input.

  python -m paper_1910_10391_gb300.surrogate --train 200000 --heldout 4096
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import time

import numpy as np

from . import _binding as rad
from . import inputs as I


@dataclasses.dataclass
class Config:
    n_omega: int = 256
    n_side: int = 32
    n_rbins: int = 8
    n_samples: int = 8192
    length: float = 100e-6
    U0_eV: float = 20.0
    d_p: float = I.SI110_DP
    gamma_lo: float = 2e3
    gamma_hi: float = 4e4
    theta_frac: float = 1.5
    n_gamma_train: int = 64
    mode: int = rad.RAD_SPIN_HALF
    precision: int = rad.RAD_MIXED
    width: int = 256
    depth: int = 3
    n_models: int = 4
    batch: int = 1024
    steps: int = 20000
    lr: float = 2e-3
    lr_min: float = 1e-5
    weight_decay: float = 1e-5
    floor_rel: float = 1e-6
    fallback_rel: float = 0.01
    chunk: int = 512
    n_fourier: int = 28
    fourier_sigma: float = 1.5
    fourier_seed: int = 11
    n_val: int = 2048
    calib_quantile: float = 0.95

    @property
    def n_in(self):
        return 6 + 2 * self.n_fourier

    @property
    def n_out(self):
        return self.n_omega * self.n_rbins


def grid_for_gamma(cfg: Config, gamma: float):
    E = gamma * I.ME_EV
    thL = math.sqrt(2.0 * cfg.U0_eV / E)
    tmax = thL + 3.0 / gamma
    hw = I.omega_log(cfg.n_omega, 1e-4 * E, 0.5 * E)
    nx, ny = cfg.n_side, cfg.n_side // 2
    d = 2.0 * tmax / cfg.n_side
    tx = -tmax + (np.arange(nx) + 0.5) * d
    ty = (np.arange(ny) + 0.5) * d
    TX, TY = np.meshgrid(tx, ty, indexing="xy")
    tx, ty = TX.ravel(), TY.ravel()
    dom = np.full(tx.size, 2.0 * d * d)  # the mirrored theta_y < 0 half
    boa = I.radial_bins(tx, ty, cfg.n_rbins, tmax)
    return I.Grid(hw, tx, ty, dom), boa, thL


def sample_entries(cfg: Config, n: int, seed: int, discrete_gamma: bool):
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(0.0, 1.0, n)
    th = rng.uniform(-cfg.theta_frac, cfg.theta_frac, n)
    lo, hi = math.log(cfg.gamma_lo), math.log(cfg.gamma_hi)
    if discrete_gamma:
        levels = np.exp(np.linspace(lo, hi, cfg.n_gamma_train))
        g = levels[rng.integers(0, cfg.n_gamma_train, n)]
    else:
        g = np.exp(rng.uniform(lo, hi, n))
    return x0, th, g


def first_line_over_E(cfg: Config, u, v, g):
    """hw1/E of the on-axis first harmonic of the transverse motion (closed form, harmonic well)."""
    E = g * I.ME_EV
    thL = np.sqrt(2.0 * cfg.U0_eV / E)
    eps = u ** 2 + (cfg.theta_frac * v) ** 2
    over = eps > 1.0
    es = np.where(over, eps, 2.0)                     # placeholder keeps arcsin defined below
    asn = np.arcsin(1.0 / np.sqrt(es))
    omega = np.where(over, 2.0 * np.pi * thL / (cfg.d_p * asn), 2.0 * thL / cfg.d_p)
    v2 = np.where(over, thL ** 2 * (np.sqrt(np.maximum(es - 1.0, 0.0)) + es * asn) / asn, 0.5 * thL ** 2 * eps)
    return 2.0 * g ** 2 * I.HBARC_EV_M * omega / (1.0 + g ** 2 * v2) / E


def grid_steps(cfg: Config, ratio):
    """Position of hw/E = ratio on the log grid, in grid steps from its first point."""
    step = math.log(0.5 / 1e-4) / (cfg.n_omega - 1)
    return np.log(ratio / 1e-4) / step


def alignment(cfg: Config, uvw, g):
    """(integer shift, fractional remainder) of each entry's first line on the photon-energy grid."""
    pos = grid_steps(cfg, first_line_over_E(cfg, uvw[:, 0], uvw[:, 1], g))
    sh = np.rint(pos).astype(np.int64)
    return sh, pos - sh


def shift_range(cfg: Config):
    """Smallest and largest shift over the input domain (dense scan of eps and gamma)."""
    ee = np.linspace(0.0, 1.0 + cfg.theta_frac ** 2, 801)
    gg = np.exp(np.linspace(math.log(cfg.gamma_lo), math.log(cfg.gamma_hi), 201))
    E2, G2 = np.meshgrid(ee, gg)
    u = np.sqrt(E2.ravel())
    v = np.zeros_like(u)
    sh = np.rint(grid_steps(cfg, first_line_over_E(cfg, u, v, G2.ravel()))).astype(np.int64)
    return int(sh.min()) - 1, int(sh.max()) + 1


def gamma_of(cfg: Config, w):
    lo, hi = math.log(cfg.gamma_lo), math.log(cfg.gamma_hi)
    return np.exp(lo + 0.5 * (np.asarray(w) + 1.0) * (hi - lo))


def raw_inputs(cfg: Config, x0, th, g):
    """(u, v, w) in [-1, 1]: 2 x0/d_p - 1, theta0/(theta_frac theta_L), scaled log gamma."""
    lo, hi = math.log(cfg.gamma_lo), math.log(cfg.gamma_hi)
    return np.stack([2.0 * x0 - 1.0, th / cfg.theta_frac, 2.0 * (np.log(g) - lo) / (hi - lo) - 1.0], 1)


def feature_map(cfg: Config, uvw):
    """Fixed map of the three inputs to the network's first layer: (u, v, w), the transverse
    energy in units of the well depth eps = u^2 + (theta_frac v)^2 (harmonic well: U = U0 u^2),
    log(eps) (spectra scale with eps for small amplitudes), and random Fourier features
    sin/cos(2 pi B (u, v, w)) with B ~ N(0, sigma^2) fixed by a seed (Tancik et al., NeurIPS 2020)."""
    uvw = np.asarray(uvw, dtype=np.float64)
    eps = uvw[:, 0] ** 2 + (cfg.theta_frac * uvw[:, 1]) ** 2
    _, frac = alignment(cfg, uvw, gamma_of(cfg, uvw[:, 2]))
    B = np.random.default_rng(cfg.fourier_seed).normal(0.0, cfg.fourier_sigma, (cfg.n_fourier, 3))
    z = 2.0 * np.pi * uvw @ B.T
    f = np.concatenate([uvw, eps[:, None] / 3.0, np.log(eps + 1e-4)[:, None] / 5.0, frac[:, None],
                        np.sin(z), np.cos(z)], 1)
    return f.astype(np.float32)


def features(cfg: Config, x0, th, g):
    return feature_map(cfg, raw_inputs(cfg, x0, th, g))


def mirrored_inputs(uvw):
    """Entry (x0, theta0) and its mirror image about the channel centre (d_p - x0, -theta0) give
    trajectories x and d_p - x: the same spectrum in every radial bin."""
    m = np.array(uvw, dtype=np.float64, copy=True)
    m[:, 0] = -m[:, 0]
    m[:, 1] = -m[:, 1]
    return m


def kernel_bins(cfg: Config, x0, th, g, stream=None):
    """Exact per-particle bins [n][n_omega][n_rbins] (device float64), grouped by gamma."""
    import torch
    n = len(x0)
    out = torch.empty((n, cfg.n_omega, cfg.n_rbins), dtype=torch.float64, device="cuda")
    dt = cfg.length / (cfg.n_samples - 1)
    order = np.argsort(g, kind="stable")
    gs = g[order]
    starts = np.flatnonzero(np.r_[True, gs[1:] != gs[:-1]])
    ends = np.r_[starts[1:], n]
    for a, b in zip(starts, ends):
        gamma = float(gs[a])
        grid, boa, thL = grid_for_gamma(cfg, gamma)
        d_hw = torch.from_numpy(grid.hbar_omega_eV).cuda()
        d_tx, d_ty = torch.from_numpy(grid.theta_x).cuda(), torch.from_numpy(grid.theta_y).cuda()
        d_dom = torch.from_numpy(grid.d_omega).cuda()
        d_boa = torch.from_numpy(boa).cuda()
        for c0 in range(a, b, cfg.chunk):
            idx = order[c0:min(b, c0 + cfg.chunk)]
            tr = I.channeling_given(x0[idx] * cfg.d_p, th[idx] * thL, np.full(len(idx), gamma), cfg.n_samples, dt,
                                    charge=+1, U0_eV=cfg.U0_eV, d_p=cfg.d_p, ms=False)
            inp = rad.DeviceInputs(tr, grid)
            w = torch.ones(len(idx), dtype=torch.float64, device="cuda")
            o = torch.empty((len(idx), cfg.n_omega, cfg.n_rbins), dtype=torch.float64, device="cuda")
            rc = rad.rad_spectrum_particles(inp.samples, inp.offsets, inp.gamma, inp.energy, w, d_hw, d_tx, d_ty,
                                            d_dom, cfg.mode, cfg.precision, None, d_boa, cfg.n_rbins, o, stream)
            if rc:
                raise rad.RadError(rc, "rad_spectrum_particles")
            out[torch.from_numpy(idx).cuda()] = o
    return out


class Surrogate:
    """Ensemble of MLPs predicting aligned log10 spectra; see the module docstring."""

    def __init__(self, cfg: Config):
        self.cfg = cfg
        self.models = []
        self.mu = self.sigma = None
        self.floor = None
        self.calib = 1.0
        self.s_lo, self.s_hi = shift_range(cfg)
        self.n_ext = cfg.n_omega + (self.s_hi - self.s_lo)

    def _window_index(self, uvw, device):
        """Column indices [n][n_out] of each entry's own 256 x 8 window in the extended output."""
        import torch
        sh, _ = alignment(self.cfg, uvw, gamma_of(self.cfg, uvw[:, 2]))
        off_np = np.clip(self.s_hi - sh, 0, self.s_hi - self.s_lo).astype(np.int64)
        off = torch.from_numpy(off_np).to(device) * self.cfg.n_rbins
        return off[:, None] + torch.arange(self.cfg.n_out, device=device)[None, :]

    def fit(self, uvw, bins_dev, val_uvw=None, val_bins=None, log=None):
        """Train the ensemble on raw inputs uvw [n][3] and their per-particle bins; a validation
        set (entries the ensemble does not train on) calibrates the error estimate."""
        import torch
        cfg = self.cfg
        n = uvw.shape[0]
        self.floor = float(bins_dev.max().item()) * cfg.floor_rel
        y = torch.empty((n, cfg.n_out), dtype=torch.float32, device="cuda")
        rad.rad_log_targets(bins_dev.reshape(-1).contiguous(), self.floor, y.view(-1))
        self.mu, self.sigma = float(y.mean().item()), float(y.std().item())
        y = (y - self.mu) / self.sigma
        # aligned targets and masks on the extended grid, for the entries and their mirror images
        uvw2 = np.concatenate([uvw, mirrored_inputs(uvw)])
        x = torch.from_numpy(feature_map(cfg, uvw2)).cuda()
        idx = self._window_index(uvw2, "cuda")
        n2 = uvw2.shape[0]
        n_ext_out = self.n_ext * cfg.n_rbins
        yt = torch.zeros((n2, n_ext_out), dtype=torch.float32, device="cuda")
        mk = torch.zeros((n2, n_ext_out), dtype=torch.float32, device="cuda")
        yt.scatter_(1, idx, torch.cat([y, y]))
        mk.scatter_(1, idx, torch.ones((n2, cfg.n_out), dtype=torch.float32, device="cuda"))
        del y
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        bsz = min(cfg.batch, n2)
        per_epoch = max(n2 // bsz, 1)
        history = []
        for k in range(cfg.n_models):
            m = rad.MLP(cfg.n_in, cfg.width, cfg.depth, n_ext_out, bsz, seed=1000 + k)
            gen = torch.Generator(device="cuda")
            gen.manual_seed(77 + k)
            perm = None
            for step in range(cfg.steps):
                if step % per_epoch == 0:
                    perm = torch.randperm(n2, device="cuda", generator=gen)
                j = step % per_epoch
                b = perm[j * bsz:(j + 1) * bsz]
                lr = cfg.lr_min + 0.5 * (cfg.lr - cfg.lr_min) * (1 + math.cos(math.pi * step / cfg.steps))
                m.train_step(x[b].contiguous(), yt[b].contiguous(), lr, cfg.weight_decay, loss,
                             mask=mk[b].contiguous())
                if step == 0 or (step + 1) % max(cfg.steps // 20, 1) == 0:
                    history.append((k, step, float(loss.item())))
                    if log:
                        log(f"model {k} step {step} loss {history[-1][2]:.5f}")
            self.models.append(m)
        del yt, mk
        # calibration: scale of the ensemble spread so that it covers the actual relative error of
        # calib_quantile of the validation entries
        self.calib = 1.0
        if val_uvw is not None and len(val_uvw) > 0 and len(self.models) > 1:
            mean, spread = self.predict(val_uvw, calibrated=False)
            nv = len(val_uvw)
            actual = rel_l2(torch.pow(10.0, mean.double()).cpu().numpy(), val_bins.reshape(nv, -1).cpu().numpy())
            ratio = actual / np.maximum(spread.cpu().numpy(), 1e-12)
            self.calib = float(np.quantile(ratio, cfg.calib_quantile))
        return history

    def predict(self, uvw, calibrated=True):
        """(log10 bins mean [n][n_out], relative error estimate [n]) as device tensors."""
        import torch
        cfg = self.cfg
        uvw = np.asarray(uvw, dtype=np.float64)
        x = torch.from_numpy(feature_map(cfg, uvw)).cuda()
        n = x.shape[0]
        idx = self._window_index(uvw, "cuda")
        ext = torch.empty((n, self.n_ext * cfg.n_rbins), dtype=torch.float32, device="cuda")
        preds = torch.empty((len(self.models), n, cfg.n_out), dtype=torch.float32, device="cuda")
        for k, m in enumerate(self.models):
            m.forward(x, ext)
            torch.gather(ext, 1, idx, out=preds[k])
        preds.mul_(self.sigma).add_(self.mu)
        mean = torch.empty((n, cfg.n_out), dtype=torch.float32, device="cuda")
        err = torch.empty(n, dtype=torch.float32, device="cuda")
        rad.rad_mlp_ensemble_estimate(preds, mean, err)
        if calibrated:
            err *= self.calib
        return mean, err

    def close(self):
        for m in self.models:
            m.close()
        self.models = []


def rel_l2(pred, truth):
    """Relative L2 error per entry over the bins within 1e-3 of the entry's maximum."""
    sig = truth >= 1e-3 * truth.max(axis=1, keepdims=True)
    return np.sqrt(((pred - truth) ** 2 * sig).sum(1) / np.maximum((truth ** 2 * sig).sum(1), 1e-300))


def evaluate(sur: Surrogate, x0, th, g, log=None):
    """Surrogate with fallback vs the exact kernel on held-out entries; returns a report dict."""
    import torch
    cfg = sur.cfg
    xf = raw_inputs(cfg, x0, th, g)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    truth = kernel_bins(cfg, x0, th, g)
    torch.cuda.synchronize()
    t_kernel = time.perf_counter() - t0

    sur.predict(xf[:1])  # warm-up (first-call costs are not part of the steady state)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mean, err = sur.predict(xf)
    err_np = err.cpu().numpy()
    t_predict = time.perf_counter() - t0
    fb = np.flatnonzero(err_np > cfg.fallback_rel)
    pred = torch.pow(10.0, mean.double()).view(-1, cfg.n_omega, cfg.n_rbins)
    if fb.size:
        pred[torch.from_numpy(fb).cuda()] = kernel_bins(cfg, x0[fb], th[fb], g[fb])
    torch.cuda.synchronize()
    t_sur = time.perf_counter() - t0

    tr = truth.cpu().numpy().reshape(len(x0), -1)
    pr = pred.cpu().numpy().reshape(len(x0), -1)
    sur_only = (10.0 ** mean.double().cpu().numpy()).reshape(len(x0), -1)
    err_sur = rel_l2(sur_only, tr)
    err_merged = rel_l2(pr, tr)
    ens_t, ens_p = tr.mean(0), pr.mean(0)
    s_ens = ens_t >= 1e-3 * ens_t.max()
    ens_err = np.abs(ens_p - ens_t)[s_ens] / ens_t[s_ens]
    # calibration: fraction of entries whose estimate is at least their actual error
    calibrated = float(np.mean(err_np >= err_sur))
    report = {
        "heldout": int(len(x0)), "fallback_fraction": float(fb.size / len(x0)),
        "rel_l2_surrogate_median": float(np.median(err_sur)), "rel_l2_surrogate_p90": float(np.quantile(err_sur, 0.9)),
        "rel_l2_merged_max": float(err_merged.max()), "rel_l2_merged_median": float(np.median(err_merged)),
        "rel_l2_merged_p99": float(np.quantile(err_merged, 0.99)), "calibration_factor": sur.calib,
        "estimate_covers_error_fraction": calibrated,
        "ensemble_spectrum_max_rel_err": float(ens_err.max()), "ensemble_spectrum_mean_rel_err": float(ens_err.mean()),
        "t_kernel_s": t_kernel, "t_predict_s": t_predict, "t_surrogate_with_fallback_s": t_sur,
        "gain": t_kernel / t_sur,
        "spectra_per_s_kernel": len(x0) / t_kernel, "spectra_per_s_surrogate": len(x0) / t_sur,
    }
    if log:
        log(json.dumps(report))
    return report


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=200000)
    ap.add_argument("--heldout", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--models", type=int, default=4)
    ap.add_argument("--n-gamma", type=int, default=64)
    ap.add_argument("--quiet", action="store_true")
    a = ap.parse_args(argv)
    import torch
    cfg = Config(steps=a.steps, n_models=a.models, n_gamma_train=a.n_gamma)
    log = (lambda s: None) if a.quiet else (lambda s: print(s, flush=True))
    x0, th, g = sample_entries(cfg, a.train, seed=5, discrete_gamma=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bins = kernel_bins(cfg, x0, th, g)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    terms = a.train * cfg.n_samples * cfg.n_omega * (cfg.n_side * cfg.n_side // 2)
    log(json.dumps({"data_s": t_data, "terms": terms, "terms_per_s": terms / t_data}))
    vx0, vth, vg = sample_entries(cfg, cfg.n_val, seed=7, discrete_gamma=False)
    vbins = kernel_bins(cfg, vx0, vth, vg)
    sur = Surrogate(cfg)
    t0 = time.perf_counter()
    hist = sur.fit(raw_inputs(cfg, x0, th, g), bins, raw_inputs(cfg, vx0, vth, vg), vbins,
                   log=None if a.quiet else log)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    del bins
    hx0, hth, hg = sample_entries(cfg, a.heldout, seed=6, discrete_gamma=False)
    rep = evaluate(sur, hx0, hth, hg)
    rep.update({"train": a.train, "steps": cfg.steps, "models": cfg.n_models, "fit_s": t_fit, "data_s": t_data,
                "final_losses": [h[2] for h in hist if h[1] == cfg.steps - 1],
                "first_losses": [h[2] for h in hist if h[1] == 0]})
    print(json.dumps(rep))
    st = rad.rad_device_status(1)
    if st:
        raise rad.RadError(st, "device status")
    sur.close()


if __name__ == "__main__":
    main()
