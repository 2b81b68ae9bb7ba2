"""Learned surrogate for per-particle planar-channeling spectra, with the exact kernel as fallback.

Entry conditions (x0/d_p, theta0/theta_L, gamma) of a positron in the harmonic planar well
(no multiple scattering, 100 um, 8192 samples) map to log10 of its spectrum dI/d(hw) in 8
radial bins of the emission angle, at 256 photon energies hw/E log-spaced in [1e-4, 0.5]
(BCK spin-1/2 model). Training spectra come from rad_spectrum_particles; the network (3 ->
256 -> 256 -> 256 -> 2048, GELU) is trained with the library's own BF16 tensor-core kernels.
An ensemble of networks gives error estimates: per entry (entries whose estimate exceeds
`fallback_rel` are recomputed with the exact kernel), and for the weighted mean spectrum of a
beam of entries (the entries with the largest estimated error contributions are recomputed with
the kernel until the mean's estimate is at most `fallback_rel`). Both estimates are calibrated,
per bin of log gamma, on validation beams the networks do not train on. Entries with transverse
energy above `eps_gate` (near or over the barrier, where plane crossings change the spectrum's
character) always take the kernel. The loss weights each output by the square of its value
relative to the entry's maximum (plus a floor): to first order that is the relative L2 error of
the spectrum that the log-space error causes.

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

  python -m paper_1910_10391_gb300.surrogate --train 200000 --heldout 4096 --beams 16 --steps 40000
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
    calib_quantile: float = 1.0
    calib_margin: float = 1.25
    loss_floor_w: float = 0.02
    beams_val: int = 32
    calib_subsets: int = 8
    calib_gamma_bins: int = 4
    beam_divergence: float = 0.3
    eps_gate: float = 0.9
    phase_budget: float = 65536.0

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


def sample_beams(cfg: Config, n_beams: int, per_beam: int, seed: int, divergence=None, gammas=None):
    """Beams of entries: each beam has one Lorentz factor, log-uniform in [gamma_lo, gamma_hi]
    (or the given `gammas`, one per beam);
    its entries have x0/d_p ~ U[0, 1) and theta0/theta_L ~ N(0, divergence^2) clipped to
    [-theta_frac, theta_frac] (a beam with the ensemble workloads' divergence, 0.3 theta_L), or
    ~ U[-theta_frac, theta_frac] when divergence is None (the training coverage).
    Returns (x0, theta0/theta_L, gamma, beam index) per entry."""
    rng = np.random.default_rng(seed)
    lo, hi = math.log(cfg.gamma_lo), math.log(cfg.gamma_hi)
    gb = np.exp(rng.uniform(lo, hi, n_beams))
    if gammas is not None:
        gb = np.asarray(gammas, dtype=np.float64)
        if gb.shape != (n_beams,) or np.any(gb < cfg.gamma_lo) or np.any(gb > cfg.gamma_hi):
            raise ValueError("one Lorentz factor per beam, inside the input domain")
    n = n_beams * per_beam
    x0 = rng.uniform(0.0, 1.0, n)
    if divergence is None:
        th = rng.uniform(-cfg.theta_frac, cfg.theta_frac, n)
    else:
        th = np.clip(rng.normal(0.0, divergence, n), -cfg.theta_frac, cfg.theta_frac)
    beam = np.repeat(np.arange(n_beams), per_beam)
    return x0, th, gb[beam], beam


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


def transverse_energy(cfg: Config, uvw):
    """Transverse energy in units of the well depth, eps = u^2 + (theta_frac v)^2 (eps > 1: over
    the barrier)."""
    uvw = np.asarray(uvw, dtype=np.float64)
    return uvw[:, 0] ** 2 + (cfg.theta_frac * uvw[:, 1]) ** 2


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


_PLANS = {}


def _plan(cfg: Config, n: int, n_angles: int):
    """Per-particle plan (radial bins) for n entries. The kernel's error is judged against the
    surrogate's 1 % contract, so mixed-precision plans take a phase budget above the library's
    default: the widest grids (gamma = 2000, theta up to theta_L + 3/gamma, hw up to E/2) reach
    in-tile phase offsets of about 2.8e4 rad, where the kernel's error is still about 1e-4."""
    key = (n, n_angles, cfg.n_omega, cfg.n_samples, cfg.n_rbins, cfg.mode, cfg.precision)
    if key not in _PLANS:
        p = rad.Plan(n * cfg.n_samples, n, cfg.n_omega, n_angles, cfg.mode, cfg.precision,
                     rad.RAD_PER_PARTICLE | 4, cfg.n_rbins)
        if cfg.precision == rad.RAD_MIXED:
            rc = p.set_phase_budget(cfg.phase_budget)
            if rc:
                raise rad.RadError(rc, "rad_plan_set_phase_budget")
        _PLANS[key] = p
    return _PLANS[key]


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
            m = len(idx)
            # pad to a multiple of 32 entries (repeating the last) so that the library sees a
            # bounded set of batch shapes and reuses their plans
            pad = np.concatenate([idx, np.full((-m) % 32, idx[-1])])
            tr = I.channeling_given(x0[pad] * cfg.d_p, th[pad] * thL, np.full(len(pad), gamma), cfg.n_samples, dt,
                                    charge=+1, U0_eV=cfg.U0_eV, d_p=cfg.d_p, ms=False)
            inp = rad.DeviceInputs(tr, grid)
            w = torch.ones(len(pad), dtype=torch.float64, device="cuda")
            o = torch.empty((len(pad), cfg.n_omega, cfg.n_rbins), dtype=torch.float64, device="cuda")
            rc = _plan(cfg, len(pad), grid.n_angles).execute(inp.samples, inp.offsets, inp.gamma, inp.energy, w,
                                                             d_hw, d_tx, d_ty, d_dom, None, None, d_boa, o,
                                                             stream=stream)
            if rc:
                raise rad.RadError(rc, "rad_plan_execute")
            out[torch.from_numpy(idx).cuda()] = o[:m]
    return out


class Surrogate:
    """Ensemble of MLPs predicting aligned log10 spectra; see the module docstring."""

    def __init__(self, cfg: Config):
        self.cfg = cfg
        self.models = []
        self.mu = self.sigma = None
        self.floor = None
        self.calib = np.ones(cfg.calib_gamma_bins)
        self.calib_ens = np.ones(cfg.calib_gamma_bins)
        self.s_lo, self.s_hi = shift_range(cfg)
        self.n_ext = cfg.n_omega + (self.s_hi - self.s_lo)

    def _window_index(self, uvw, device):
        """Column indices [n][n_out] of each entry's own 256 x 8 window in the extended output."""
        import torch
        sh, _ = alignment(self.cfg, uvw, gamma_of(self.cfg, uvw[:, 2]))
        off_np = np.clip(self.s_hi - sh, 0, self.s_hi - self.s_lo).astype(np.int64)
        off = torch.from_numpy(off_np).to(device) * self.cfg.n_rbins
        return off[:, None] + torch.arange(self.cfg.n_out, device=device)[None, :]

    def gamma_bin(self, g):
        """Calibration bin of Lorentz factors g: equal widths in log gamma over the input domain."""
        cfg = self.cfg
        lo, hi = math.log(cfg.gamma_lo), math.log(cfg.gamma_hi)
        b = np.floor((np.log(np.asarray(g, dtype=np.float64)) - lo) / (hi - lo) * cfg.calib_gamma_bins)
        return np.clip(b, 0, cfg.calib_gamma_bins - 1).astype(np.int64)

    def fit(self, uvw, bins_dev, val_uvw=None, val_bins=None, val_beam=None, log=None):
        """Train the ensemble on raw inputs uvw [n][3] and their per-particle bins; a validation
        set (entries the ensemble does not train on, grouped in beams by val_beam) calibrates the
        per-entry and the beam-mean error estimates."""
        import torch
        cfg = self.cfg
        n = uvw.shape[0]
        self.floor = float(bins_dev.max().item()) * cfg.floor_rel
        y = torch.empty((n, cfg.n_out), dtype=torch.float32, device="cuda")
        rad.rad_log_targets(bins_dev.reshape(-1).contiguous(), self.floor, y.view(-1))
        self.mu, self.sigma = float(y.mean().item()), float(y.std().item())
        y = (y - self.mu) / self.sigma
        flat = bins_dev.reshape(n, -1)
        wt = (flat / flat.amax(1, keepdim=True).clamp_min(1e-300)).pow(2).add_(cfg.loss_floor_w).float()
        # aligned targets and masks on the extended grid, for the entries and their mirror images
        uvw2 = np.concatenate([uvw, mirrored_inputs(uvw)])
        x = torch.from_numpy(feature_map(cfg, uvw2)).cuda()
        idx = self._window_index(uvw2, "cuda")
        n2 = uvw2.shape[0]
        n_ext_out = self.n_ext * cfg.n_rbins
        yt = torch.zeros((n2, n_ext_out), dtype=torch.float32, device="cuda")
        mk = torch.zeros((n2, n_ext_out), dtype=torch.float32, device="cuda")
        yt.scatter_(1, idx, torch.cat([y, y]))
        mk.scatter_(1, idx, torch.cat([wt, wt]))
        del y, wt
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
        # calibration, per bin of log gamma: scales of the ensemble spreads so that they cover the
        # actual relative errors of calib_quantile of the validation entries, and of validation
        # beam means (every beam and half-size subsets of it); a bin with too few validation
        # beams takes the largest factor of the other bins
        nb = cfg.calib_gamma_bins
        self.calib = np.ones(nb)
        self.calib_ens = np.ones(nb)
        if val_uvw is not None and len(val_uvw) > 0 and len(self.models) > 1:
            nv = len(val_uvw)
            members = self.members(val_uvw)
            mean, spread = self._estimate(members)
            served = torch.pow(10.0, mean.double())
            truth = val_bins.reshape(nv, -1)
            actual = rel_l2(served.cpu().numpy(), truth.cpu().numpy())
            ratio = actual / np.maximum(spread.cpu().numpy(), 1e-12)
            gb = self.gamma_bin(gamma_of(cfg, np.asarray(val_uvw)[:, 2]))
            glob = float(np.quantile(ratio, cfg.calib_quantile))
            for k in range(nb):
                sel = gb == k
                self.calib[k] = np.quantile(ratio[sel], cfg.calib_quantile) if sel.sum() >= 20 else np.nan
            self.calib = np.where(np.isnan(self.calib), max(glob, float(np.nanmax(np.r_[self.calib, glob]))),
                                  self.calib)
            if val_beam is not None:
                # the policy's estimate after fallback of the first j entries (gated ones first,
                # then by estimated contribution), against the actual error of that mean, at
                # several fallback depths from "gated entries only" to most of the beam
                rng = np.random.default_rng(cfg.fourier_seed + 1)
                ratios = [[] for _ in range(nb)]
                gated_all = transverse_energy(cfg, val_uvw) > cfg.eps_gate
                ce_all = torch.from_numpy(self.calib[gb]).cuda() * spread.double()
                for b in np.unique(val_beam):
                    sel = np.flatnonzero(val_beam == b)
                    k = int(gb[sel[0]])
                    for j in range(cfg.calib_subsets):
                        sub = sel if j == 0 else np.sort(rng.choice(sel, size=max(len(sel) // 2, 2), replace=False))
                        gsub = gated_all[sub]
                        m = len(sub)
                        j0 = int(gsub.sum())
                        if j0 == m:
                            continue
                        st = torch.from_numpy(sub).cuda()
                        w = torch.full((m,), 1.0 / m, dtype=torch.float64, device="cuda")
                        sv, tv = served[st], truth[st]
                        contrib = ce_all[st] * w * torch.linalg.norm(sv, dim=1)
                        contrib = torch.where(torch.from_numpy(gsub).cuda(), torch.full_like(contrib, float("inf")),
                                              contrib)
                        order = torch.argsort(contrib, descending=True)
                        curve = self._fallback_curve(members[:, st], w, order)
                        mt = (tv * w[:, None]).sum(0)
                        sig = mt >= 1e-3 * mt.max()
                        diff = ((sv - tv) * w[:, None])[order][:, sig]
                        tail = torch.flip(torch.cumsum(torch.flip(diff, [0]), 0), [0])
                        den = torch.linalg.norm(mt[sig])
                        for jj in sorted({j0 + int(f * (m - j0)) for f in (0.0, 0.1, 0.2, 0.35, 0.5, 0.7)}):
                            if jj >= m:
                                continue
                            act = float(torch.linalg.norm(tail[jj]) / den)
                            ratios[k].append(act / max(float(curve[jj]), 1e-12))
                glob = float(np.quantile(np.concatenate([np.asarray(r) for r in ratios]), cfg.calib_quantile))
                self.calib_ens = np.array([np.quantile(r, cfg.calib_quantile) if len(r) >= 3 * cfg.calib_subsets
                                           else np.nan for r in ratios])
                fill = max(glob, float(np.nanmax(np.r_[self.calib_ens, glob])))
                self.calib_ens = np.where(np.isnan(self.calib_ens), fill, self.calib_ens)
            # the validation set is finite: a margin over the largest ratio seen covers beams whose
            # ratio lies beyond it
            self.calib = self.calib * cfg.calib_margin
            self.calib_ens = self.calib_ens * cfg.calib_margin
        return history

    def members(self, uvw):
        """log10 bins of every model [n_models][n][n_out] (device float32)."""
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
        return preds.mul_(self.sigma).add_(self.mu)

    def _estimate(self, members):
        import torch
        n = members.shape[1]
        mean = torch.empty((n, self.cfg.n_out), dtype=torch.float32, device="cuda")
        err = torch.empty(n, dtype=torch.float32, device="cuda")
        rad.rad_mlp_ensemble_estimate(members, mean, err)
        return mean, err

    def _fallback_curve(self, members, w, order):
        """Uncalibrated relative error estimate of the weighted mean spectrum when the first j
        entries of `order` come from the kernel, for j = 0..n: the L2 norm of the models' spread
        (standard deviation over models) of the remaining entries' weighted sum, over the L2
        norm of the mean spectrum."""
        import torch
        lin = torch.pow(10.0, members[:, order].double()) * w[order][None, :, None]
        tail = torch.flip(torch.cumsum(torch.flip(lin, [1]), 1), [1])     # tail[:, j] = sum over i >= j
        sd = torch.cat([tail.var(0, unbiased=True).sum(1), tail.new_zeros(1)]).sqrt_()
        served = (torch.pow(10.0, members.double().mean(0)) * w[:, None]).sum(0)
        return sd / torch.linalg.norm(served).clamp_min(1e-300)

    def ensemble_average(self, x0, th, g, weight=None, fallback_rel=None):
        """Weighted mean bins [n_omega][n_rbins] (device float64) of one beam's entries and a dict
        (n_fallback, estimate, estimate_surrogate_only): surrogate predictions, with the entries of
        largest estimated error contribution recomputed by the kernel until the calibrated
        estimate of the mean's relative L2 error is at most fallback_rel."""
        import torch
        cfg = self.cfg
        bar = cfg.fallback_rel if fallback_rel is None else fallback_rel
        n = len(x0)
        w_np = np.full(n, 1.0 / n) if weight is None else np.asarray(weight, np.float64) / np.sum(weight)
        w = torch.from_numpy(w_np).cuda()
        uvw = raw_inputs(cfg, x0, th, g)
        members = self.members(uvw)
        mean, err = self._estimate(members)
        served = torch.pow(10.0, mean.double())
        ce = torch.from_numpy(self.calib[self.gamma_bin(g)]).cuda()
        contrib = err.double() * ce * w * torch.linalg.norm(served, dim=1)
        # entries near or over the barrier always take the kernel: their spectra change character
        # there (plane crossings) and the network does not reach percent accuracy on them
        gated = torch.from_numpy(transverse_energy(cfg, uvw) > cfg.eps_gate).cuda()
        contrib = torch.where(gated, torch.full_like(contrib, float("inf")), contrib)
        order = torch.argsort(contrib, descending=True)
        j0 = int(gated.sum().item())
        g_beam = float(np.exp(np.sum(w_np * np.log(g))))  # weighted geometric mean Lorentz factor
        curve = float(self.calib_ens[self.gamma_bin(g_beam)]) * self._fallback_curve(members, w, order)
        j = j0 + int(torch.nonzero(curve[j0:] <= bar)[0, 0].item())
        keep = order[j:]
        total = (served[keep] * w[keep, None]).sum(0)
        if j:
            fb = order[:j].cpu().numpy()
            exact = kernel_bins(cfg, x0[fb], th[fb], g[fb]).view(j, -1)
            total += (exact * w[order[:j], None]).sum(0)
        info = {"n_fallback": j, "estimate": float(curve[j].item()), "estimate_surrogate_only": float(curve[0].item())}
        return total.view(cfg.n_omega, cfg.n_rbins), info

    def predict(self, uvw, calibrated=True):
        """(log10 bins mean [n][n_out], relative error estimate [n]) as device tensors."""
        import torch
        mean, err = self._estimate(self.members(uvw))
        if calibrated:
            k = self.gamma_bin(gamma_of(self.cfg, np.asarray(uvw)[:, 2]))
            err *= torch.from_numpy(self.calib[k].astype(np.float32)).cuda()
        return mean, err

    def close(self):
        for m in self.models:
            m.close()
        self.models = []


def rel_l2(pred, truth):
    """Relative L2 error per entry over the bins within 1e-3 of the entry's maximum."""
    sig = truth >= 1e-3 * truth.max(axis=1, keepdims=True)
    return np.sqrt(((pred - truth) ** 2 * sig).sum(1) / np.maximum((truth ** 2 * sig).sum(1), 1e-300))


def evaluate(sur: Surrogate, x0, th, g, beam, log=None):
    """Surrogate with fallback vs the exact kernel on held-out beams; returns a report dict.

    Per entry: the surrogate's relative L2 error, its calibrated estimate, and the merged result
    with per-entry fallback. Per beam: the uniform-weight mean spectrum from ensemble_average
    (fallback until the estimate is at most fallback_rel) against the kernel's, with the time
    of each path; gain = kernel time / surrogate-with-fallback time over all beams."""
    import torch
    cfg = sur.cfg
    beams = np.unique(beam)
    # warm-up of every step on two entries (first-call costs are not steady state)
    kernel_bins(cfg, x0[:2], th[:2], g[:2])
    sur.ensemble_average(x0[:2], th[:2], g[:2], fallback_rel=0.0)
    truth = torch.empty((len(x0), cfg.n_omega, cfg.n_rbins), dtype=torch.float64, device="cuda")
    t_kernel, t_sur, ens = [], [], []
    for b in beams:
        sel = np.flatnonzero(beam == b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        truth[torch.from_numpy(sel).cuda()] = kernel_bins(cfg, x0[sel], th[sel], g[sel])
        torch.cuda.synchronize()
        t_kernel.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        avg, info = sur.ensemble_average(x0[sel], th[sel], g[sel])
        torch.cuda.synchronize()
        t_sur.append(time.perf_counter() - t0)
        ref = truth[torch.from_numpy(sel).cuda()].mean(0).reshape(1, -1).cpu().numpy()
        info["error"] = float(rel_l2(avg.reshape(1, -1).cpu().numpy(), ref)[0])
        m_only, _ = sur.predict(raw_inputs(cfg, x0[sel], th[sel], g[sel]))
        info["error_surrogate_only"] = float(rel_l2(torch.pow(10.0, m_only.double()).mean(0, keepdim=True).cpu().numpy(),
                                                    ref)[0])
        info["gamma"] = float(g[sel[0]])
        info["entries"] = int(len(sel))
        ens.append(info)

    t0 = time.perf_counter()
    mean, err = sur.predict(raw_inputs(cfg, x0, th, g))
    err_np = err.cpu().numpy()
    t_predict = time.perf_counter() - t0
    tr = truth.cpu().numpy().reshape(len(x0), -1)
    sur_only = (10.0 ** mean.double().cpu().numpy()).reshape(len(x0), -1)
    err_sur = rel_l2(sur_only, tr)
    fb = (err_np > cfg.fallback_rel) | (transverse_energy(cfg, raw_inputs(cfg, x0, th, g)) > cfg.eps_gate)
    merged = np.where(fb[:, None], tr, sur_only)
    err_merged = rel_l2(merged, tr)
    e_err = np.array([e["error"] for e in ens])
    eps = (2.0 * x0 - 1.0) ** 2 + th ** 2
    by_eps = {}
    for lo, hi in ((0.0, 0.5), (0.5, 0.9), (0.9, 1.1), (1.1, 10.0)):
        sel = (eps >= lo) & (eps < hi)
        if sel.any():
            by_eps[f"{lo}-{hi}"] = [int(sel.sum()), float(np.median(err_sur[sel])), float(np.quantile(err_sur[sel], 0.9))]
    gbin = sur.gamma_bin(g)
    by_gamma = {int(k): [int((gbin == k).sum()), float(np.median(err_sur[gbin == k]))] for k in np.unique(gbin)}
    e_est = np.array([e["estimate"] for e in ens])
    n_fb = sum(e["n_fallback"] for e in ens)
    report = {
        "heldout": int(len(x0)), "beams": int(len(beams)), "fallback_rel": cfg.fallback_rel,
        "calibration_factor": [float(c) for c in sur.calib], "calibration_factor_mean": [float(c) for c in sur.calib_ens],
        "entry_rel_l2_by_eps": by_eps, "entry_rel_l2_by_gamma_bin": by_gamma,
        "mean_error_surrogate_only_median": float(np.median([e["error_surrogate_only"] for e in ens])),
        "mean_error_surrogate_only_max": float(np.max([e["error_surrogate_only"] for e in ens])),
        "entry_rel_l2_surrogate_median": float(np.median(err_sur)),
        "entry_rel_l2_surrogate_p90": float(np.quantile(err_sur, 0.9)),
        "entry_estimate_covers_error_fraction": float(np.mean(err_np >= err_sur)),
        "entry_fallback_fraction": float(fb.mean()), "entry_rel_l2_merged_max": float(err_merged.max()),
        "mean_error_max": float(e_err.max()), "mean_error_median": float(np.median(e_err)),
        "mean_estimate_max": float(e_est.max()),
        "mean_estimate_covers_error_fraction": float(np.mean(e_est >= e_err)),
        "mean_surrogate_only_estimate_median": float(np.median([e["estimate_surrogate_only"] for e in ens])),
        "mean_fallback_fraction": float(n_fb / len(x0)),
        "t_kernel_s": float(sum(t_kernel)), "t_surrogate_with_fallback_s": float(sum(t_sur)),
        "t_predict_all_s": t_predict, "gain": float(sum(t_kernel) / sum(t_sur)),
        "spectra_per_s_kernel": len(x0) / sum(t_kernel), "spectra_per_s_surrogate": len(x0) / sum(t_sur),
        "per_beam": ens,
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
    ap.add_argument("--beams", type=int, default=16)
    ap.add_argument("--edge-beams", type=int, default=4,
                    help="of the held-out beams, this many at the ends of the Lorentz-factor range")
    ap.add_argument("--save", default="")
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
    vx0, vth, vg, vbeam = sample_beams(cfg, cfg.beams_val, cfg.n_val // cfg.beams_val, seed=7,
                                       divergence=cfg.beam_divergence)
    vbins = kernel_bins(cfg, vx0, vth, vg)
    sur = Surrogate(cfg)
    t0 = time.perf_counter()
    hist = sur.fit(raw_inputs(cfg, x0, th, g), bins, raw_inputs(cfg, vx0, vth, vg), vbins, vbeam,
                   log=None if a.quiet else log)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    del bins
    rng = np.random.default_rng(6)
    lo, hi = math.log(cfg.gamma_lo), math.log(cfg.gamma_hi)
    gb = np.exp(rng.uniform(lo, hi, a.beams))
    edge = [cfg.gamma_lo * 1.02, cfg.gamma_hi / 1.02, cfg.gamma_lo * 1.1, cfg.gamma_hi / 1.1]
    for k in range(min(a.edge_beams, a.beams)):
        gb[k] = edge[k % 4] * (1.0 + 0.01 * (k // 4))
    hx0, hth, hg, hbeam = sample_beams(cfg, a.beams, a.heldout // a.beams, seed=6, divergence=cfg.beam_divergence,
                                       gammas=gb)
    rep = evaluate(sur, hx0, hth, hg, hbeam)
    # per-entry accuracy over the whole training domain (uniform coverage), no fallback
    ux0, uth, ug, _ = sample_beams(cfg, 64, 16, seed=8)
    mean_u, _ = sur.predict(raw_inputs(cfg, ux0, uth, ug))
    tru = kernel_bins(cfg, ux0, uth, ug).reshape(len(ux0), -1).cpu().numpy()
    err_u = rel_l2(10.0 ** mean_u.double().cpu().numpy(), tru)
    eps_u = (2.0 * ux0 - 1.0) ** 2 + uth ** 2
    rep["coverage_entry_rel_l2"] = {
        "entries": int(len(ux0)), "median": float(np.median(err_u)),
        "median_channeled": float(np.median(err_u[eps_u < 0.9])),
        "median_over_barrier": float(np.median(err_u[eps_u > 1.1]))}
    rep.update({"train": a.train, "steps": cfg.steps, "models": cfg.n_models, "fit_s": t_fit, "data_s": t_data,
                "final_losses": [h[2] for h in hist if h[1] == cfg.steps - 1],
                "first_losses": [h[2] for h in hist if h[1] == 0]})
    print(json.dumps(rep))
    if a.save:
        with open(a.save, "w") as f:
            json.dump(rep, f, indent=1)
    st = rad.rad_device_status(1)
    if st:
        raise rad.RadError(st, "device status")
    sur.close()


if __name__ == "__main__":
    main()
