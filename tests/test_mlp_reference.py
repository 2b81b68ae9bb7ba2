"""The FP64 reference MLP (oracle/mlp.py) against central finite differences of its loss."""
import numpy as np

from oracle import mlp as M


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_in, width, depth, n_out = 3, 6, 3, 5
    _, npar = M.layout(n_in, width, depth, n_out)
    p = rng.normal(0, 0.5, npar)
    x = rng.normal(0, 1, (7, n_in))
    t = rng.normal(0, 1, (7, n_out))
    loss, g = M.loss_and_grad(p, x, t, n_in, width, depth, n_out)
    h = 1e-6
    for i in range(npar):
        e = np.zeros(npar)
        e[i] = h
        lp, _ = M.loss_and_grad(p + e, x, t, n_in, width, depth, n_out)
        lm, _ = M.loss_and_grad(p - e, x, t, n_in, width, depth, n_out)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(fd)


def test_gelu_values():
    # GELU(0) = 0, GELU(z) -> z for large z, GELU(-z) -> 0; derivative at 0 is 1/2
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert abs(M.gelu(np.array([8.0]))[0] - 8.0) < 1e-12
    assert abs(M.gelu(np.array([-8.0]))[0]) < 1e-12
    assert abs(M.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
