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
