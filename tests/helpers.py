"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and compare
with the FP64 oracle under the tolerances stated in the tests."""
import numpy as np
from scipy.special import jv

import oracle as O
import paper_1910_10391_gb300 as rad

MODE_ORC = {rad.RAD_CLASSICAL: O.CLASSICAL, rad.RAD_SPIN0: O.SPIN0, rad.RAD_SPIN_HALF: O.SPIN_HALF}


def gpu_cube(tr, grid, mode, precision, shape=None, outputs=("cube",), bin_of_angle=None, n_bins=0,
             plan=False, prepass=None, split=None):
    """Cube (and optional spectrum/bins) from the CUDA library, as numpy arrays."""
    import torch
    inp = rad.DeviceInputs(tr, grid, bin_of_angle=bin_of_angle, n_bins=n_bins)
    want = ("cube" in outputs) * 1 + ("spectrum" in outputs) * 2 + ("bins" in outputs) * 4
    oc = torch.full((inp.n_omega * inp.n_angles,), np.nan, dtype=torch.float64, device="cuda")
    os_ = torch.full((inp.n_omega,), np.nan, dtype=torch.float64, device="cuda")
    ob = torch.full((inp.n_omega * max(n_bins, 1),), np.nan, dtype=torch.float64, device="cuda")
    oc_, os2, ob_ = (oc if want & 1 else None), (os_ if want & 2 else None), (ob if want & 4 else None)
    if shape is None and not plan and prepass is None and split is None:
        rc = rad.rad_spectrum(*inp.args(), mode, precision, oc_, os2, inp.boa if want & 4 else None,
                              n_bins if want & 4 else 0, ob_, 0)
        assert rc == rad.RAD_OK, rad.rad_status_string(rc)
    else:
        p = rad.Plan(inp.n_samples, inp.n_particles, inp.n_omega, inp.n_angles, mode, precision, want,
                     n_bins if want & 4 else 0)
        if prepass is not None:
            assert p.set_prepass(prepass) == rad.RAD_OK
        if shape is not None:
            assert p.set_shape(*shape) == rad.RAD_OK, shape
        if prepass is not None:
            assert f"pp={int(bool(prepass))}" in p.describe(), p.describe()
        if split is not None:
            assert p.set_sincos_split(split) == rad.RAD_OK, split
            assert f"pe={split}" in p.describe(), p.describe()
        rc = p.execute(*inp.args(), oc_, os2, inp.boa if want & 4 else None, ob_)
        assert rc == rad.RAD_OK, rad.rad_status_string(rc)
        torch.cuda.synchronize()
        p.close()
    torch.cuda.synchronize()
    st = rad.rad_device_status(1)
    assert st == rad.RAD_OK, rad.rad_status_string(st)
    res = {}
    if want & 1:
        res["cube"] = oc.view(inp.n_omega, inp.n_angles).cpu().numpy()
    if want & 2:
        res["spectrum"] = os_.cpu().numpy()
    if want & 4:
        res["bins"] = ob.view(inp.n_omega, n_bins).cpu().numpy()
    return res


def assert_fp64_close(got, ref, rel=1e-9, floor=1e-6):
    """|got - ref| <= rel * max(|ref|, floor * peak) per element (peak = max |ref|)."""
    got, ref = np.asarray(got), np.asarray(ref)
    peak = np.abs(ref).max()
    bound = rel * np.maximum(np.abs(ref), floor * peak)
    err = np.abs(got - ref)
    bad = err > bound
    if bad.any():
        i = np.unravel_index(np.argmax(err / np.maximum(bound, 1e-300)), ref.shape)
        raise AssertionError(f"{bad.sum()} / {bad.size} elements outside tolerance; worst at {i}: "
                             f"got {got[i]!r} ref {ref[i]!r} (peak {peak:.3e})")
    return float((err / np.maximum(np.abs(ref), floor * peak)).max()) if peak > 0 else 0.0


def assert_mixed_close(got, ref, rel=1e-4, level=1e-3):
    """Relative error <= rel on elements with ref >= level * peak; returns error statistics."""
    got, ref = np.asarray(got), np.asarray(ref)
    peak = np.abs(ref).max()
    sel = np.abs(ref) >= level * peak
    r = np.abs(got[sel] - ref[sel]) / np.abs(ref[sel])
    stats = {"n": int(sel.sum()), "max": float(r.max()) if r.size else 0.0,
             "p99": float(np.quantile(r, 0.99)) if r.size else 0.0,
             "median": float(np.median(r)) if r.size else 0.0}
    assert stats["max"] <= rel, stats
    # everywhere else the absolute error stays below rel * level * peak
    assert np.all(np.abs(got - ref)[~sel] <= rel * level * peak * 10), "small bins off"
    return stats


def strong_undulator_on_axis(n, K, gamma, N):
    """Textbook on-axis line height of harmonic n of a planar undulator (classical):
    d2I/dhw dOmega = alpha N^2 gamma^2 F_n(K), F_n = n^2 K^2/(1+K^2/2)^2
    [J_{(n-1)/2}(xi) - J_{(n+1)/2}(xi)]^2 with xi = n K^2/(4 (1+K^2/2)) for odd n, 0 for even n."""
    if n % 2 == 0:
        return 0.0
    xi = n * K * K / (4 * (1 + K * K / 2))
    Fn = n * n * K * K / (1 + K * K / 2) ** 2 * (jv((n - 1) // 2, xi) - jv((n + 1) // 2, xi)) ** 2
    return O.ALPHA * N * N * gamma * gamma * Fn


def planar_undulator_exact(hw_eV, theta_x, theta_y, gamma, K, lam_u, N):
    """|I|^2 (the S of the classical model, before alpha/(4 pi^2)) of the planar undulator
    trajectory x = K/(gamma k) sin(kt), dz = -(K/gamma)^2/4 (t + sin(2kt)/(2k)) over N whole periods,
    for any photon energy, as the continuous integral of Sec. II's expanded form evaluated in
    closed form (independent of the time-domain sum):
      * by parts, f = d/dt[(n - beta)/(1 - n.beta)] and d(phase)/dt = w (1 - n.beta), so
        I = [g e^{i phase}]_0^T - i w int (n - beta) e^{i phase} dt with g = (n - beta)/(1 - n.beta);
        g is periodic and the phase gains w_bar T over whole periods, so the boundary term is
        g(0) (e^{i w_bar T} - 1);
      * phase = w_bar t + xi sin(2kt) - eta sin(kt), w_bar = w (1 + K^2/2 + gamma^2 theta^2)/(2 gamma^2),
        xi = w K^2/(8 gamma^2 k), eta = w theta_x K/(gamma k); by Jacobi-Anger
        e^{i phase} = sum_j C_j e^{i (w_bar + j k) t}, C_j = sum_m J_m(xi) J_{2m-j}(eta);
      * the transverse and longitudinal parts of n - beta are trigonometric polynomials
        (theta_x - (K/gamma) cos kt, theta_y, c0 + (K^2/(4 gamma^2)) cos 2kt with
        c0 = 1/(2 gamma^2) - theta^2/2 + K^2/(4 gamma^2)), so each integral is a sum of
        G(W) = int_0^T e^{i W t} dt.
    At a resonance (w_bar = n k) only the terms with j = -n survive and the result is the
    textbook generalized-Bessel angular-spectral density of harmonic n.
    hw_eV [n_omega], theta_x/theta_y [n_angles]; returns [n_omega][n_angles]."""
    from scipy.special import jv
    hw = np.asarray(hw_eV, np.float64)[:, None]
    tx = np.asarray(theta_x, np.float64)[None, :]
    ty = np.asarray(theta_y, np.float64)[None, :]
    k = 2.0 * np.pi / lam_u
    T = N * lam_u
    w = hw / O.HBARC_EV_M
    g2 = gamma * gamma
    th2 = tx * tx + ty * ty
    wbar = w * (1.0 + 0.5 * K * K + g2 * th2) / (2.0 * g2)
    xi = w * K * K / (8.0 * g2 * k)
    eta = w * tx * K / (gamma * k)
    mmax = int(np.ceil(np.max(xi))) + 20
    jmax = 2 * mmax + int(np.ceil(np.max(np.abs(eta)))) + 24
    m = np.arange(-mmax, mmax + 1)
    Jm = jv(m[:, None, None], xi[None, :, :] * np.ones_like(tx)[None, :, :])  # [m][i][j]
    pmax = 2 * mmax + jmax
    Jp = jv(np.arange(-pmax, pmax + 1)[:, None, None], eta[None, :, :] * np.ones_like(hw)[None, :, :])

    def C(j):
        return np.einsum("mij,mij->ij", Jm, Jp[2 * m - j + pmax])

    def G(W):
        # int_0^T e^{iWt} dt = T e^{iWT/2} sinc(WT/2), without 0/0
        return T * np.exp(0.5j * W * T) * np.sinc(W * T / (2.0 * np.pi))

    js = np.arange(-jmax, jmax + 1)
    Gs = {j: G(wbar + j * k) for j in range(-jmax - 2, jmax + 3)}
    e0 = np.zeros(wbar.shape, complex)
    c1 = np.zeros(wbar.shape, complex)
    c2 = np.zeros(wbar.shape, complex)
    for j in js:
        Cj = C(j)
        e0 += Cj * Gs[j]
        c1 += 0.5 * Cj * (Gs[j + 1] + Gs[j - 1])
        c2 += 0.5 * Cj * (Gs[j + 2] + Gs[j - 2])
    c0 = 1.0 / (2.0 * g2) - 0.5 * th2 + K * K / (4.0 * g2)
    D0 = 1.0 / (2.0 * g2) + 0.5 * th2 + K * K / (2.0 * g2) - tx * K / gamma
    ring = np.exp(1j * wbar * T) - 1.0
    Ix = (tx - K / gamma) / D0 * ring - 1j * w * (tx * e0 - (K / gamma) * c1)
    Iy = ty / D0 * ring - 1j * w * (ty * e0)
    Iz = (c0 + K * K / (4.0 * g2)) / D0 * ring - 1j * w * (c0 * e0 + (K * K / (4.0 * g2)) * c2)
    return np.abs(Ix) ** 2 + np.abs(Iy) ** 2 + np.abs(Iz) ** 2
