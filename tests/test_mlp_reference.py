"""The FP64 reference MLP (oracle/mlp.py) against central finite differences of its loss."""
import numpy as np
import pytest

from oracle import mlp as M


@pytest.mark.parametrize("weighted", [False, True])
def test_reference_gradient_matches_finite_differences(weighted):
    rng = np.random.default_rng(0)
    n_in, width, depth, n_out = 3, 6, 3, 5
    _, npar = M.layout(n_in, width, depth, n_out)
    p = rng.normal(0, 0.5, npar)
    x = rng.normal(0, 1, (7, n_in))
    t = rng.normal(0, 1, (7, n_out))
    m = np.where(rng.random((7, n_out)) < 0.6, rng.uniform(0.1, 2.0, (7, n_out)), 0.0) if weighted else None
    loss, g = M.loss_and_grad(p, x, t, n_in, width, depth, n_out, mask=m)
    h = 1e-6
    for i in range(npar):
        e = np.zeros(npar)
        e[i] = h
        lp, _ = M.loss_and_grad(p + e, x, t, n_in, width, depth, n_out, mask=m)
        lm, _ = M.loss_and_grad(p - e, x, t, n_in, width, depth, n_out, mask=m)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(fd)


def test_weighted_loss_value():
    # loss = sum m (y - t)^2 / (batch n_out), checked against a direct evaluation of the network
    rng = np.random.default_rng(2)
    n_in, width, depth, n_out = 2, 4, 2, 3
    _, npar = M.layout(n_in, width, depth, n_out)
    p = rng.normal(0, 0.5, npar)
    x, t = rng.normal(0, 1, (5, n_in)), rng.normal(0, 1, (5, n_out))
    m = rng.uniform(0, 3, (5, n_out))
    y = M.forward(p, x, n_in, width, depth, n_out)
    loss, _ = M.loss_and_grad(p, x, t, n_in, width, depth, n_out, mask=m)
    direct = sum(m[b, o] * (y[b, o] - t[b, o]) ** 2 for b in range(5) for o in range(n_out)) / 15
    assert abs(loss - direct) <= 1e-13 * direct


def test_gelu_values():
    # GELU(0) = 0, GELU(z) -> z for large z, GELU(-z) -> 0; derivative at 0 is 1/2
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert abs(M.gelu(np.array([8.0]))[0] - 8.0) < 1e-12
    assert abs(M.gelu(np.array([-8.0]))[0]) < 1e-12
    assert abs(M.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15


def test_grad_magnitudes_bound_the_gradient():
    """Triangle inequality: |gradient| <= the sum of its products' magnitudes, elementwise; equal
    for a linear model (depth 0) on one sample, where each gradient element is a single product."""
    rng = np.random.default_rng(3)
    n_in, width, depth, n_out, B = 3, 16, 2, 5, 12
    _, n_p = M.layout(n_in, width, depth, n_out)
    p = rng.normal(0, 0.5, n_p)
    x, t = rng.normal(0, 1, (B, n_in)), rng.normal(0, 1, (B, n_out))
    _, g = M.loss_and_grad(p, x, t, n_in, width, depth, n_out)
    mag = M.grad_magnitudes(p, x, t, n_in, width, depth, n_out)
    assert np.all(np.abs(g) <= mag * (1 + 1e-12))
    _, n1 = M.layout(n_in, width, 0, n_out)
    p1 = rng.normal(0, 0.5, n1)
    _, g1 = M.loss_and_grad(p1, x[:1], t[:1], n_in, width, 0, n_out)
    np.testing.assert_allclose(M.grad_magnitudes(p1, x[:1], t[:1], n_in, width, 0, n_out), np.abs(g1), rtol=1e-14)


def test_adamw_step_closed_forms():
    """AdamW against its closed forms: after the first step the bias-corrected moments are g and
    g^2, so the update is lr (g / (|g| + eps) + wd p); a constant gradient keeps m_hat = g and
    v_hat = g^2 at every step; a zero gradient leaves pure decay p (1 - lr wd)."""
    rng = np.random.default_rng(4)
    p, g = rng.normal(0, 1, 50), rng.normal(0, 1e-3, 50)
    lr, b1, b2, eps, wd = 1e-2, 0.9, 0.999, 1e-4, 0.1
    z = np.zeros(50)
    p1, m1, v1 = M.adamw_step(p, g, z, z, 1, lr, b1, b2, eps, wd)
    np.testing.assert_allclose(p1, p - lr * (g / (np.abs(g) + eps) + wd * p), rtol=1e-13)
    np.testing.assert_allclose(m1, (1 - b1) * g, rtol=1e-14)
    np.testing.assert_allclose(v1, (1 - b2) * g * g, rtol=1e-14)
    q, m, v = p.copy(), z, z
    for s in range(1, 30):
        q_prev = q
        q, m, v = M.adamw_step(q, g, m, v, s, lr, b1, b2, eps, 0.0)
        np.testing.assert_allclose(q_prev - q, lr * g / (np.abs(g) + eps), rtol=1e-9)
    q, _, _ = M.adamw_step(p, z, z, z, 1, lr, b1, b2, eps, wd)
    np.testing.assert_allclose(q, p * (1 - lr * wd), rtol=1e-15)
