"""Surrogate MLP kernels against the FP64 reference network (oracle/mlp.py)."""
import numpy as np
import pytest

import paper_1910_10391_gb300 as rad
from oracle import mlp as M

pytestmark = pytest.mark.gpu


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest even), returned as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32)


def gpu_params_for_reference(m, n_in, width, depth, n_out):
    """GPU parameters with the BF16 rounding the GEMM layers see (layer 0 stays FP32)."""
    p = m.get(0).astype(np.float64)
    lay, _ = M.layout(n_in, width, depth, n_out)
    for l, (wo, bo, fo, fi) in enumerate(lay):
        if l > 0:
            p[wo:wo + fo * fi] = bf16_round(p[wo:wo + fo * fi])
    return p


def test_forward_and_gradients_match_reference():
    import torch
    rng = np.random.default_rng(1)
    n_in, width, depth, n_out, B = 3, 64, 3, 96, 48
    m = rad.MLP(n_in, width, depth, n_out, max_batch=64, seed=3)
    x = rng.uniform(-1, 1, (B, n_in)).astype(np.float32)
    t = rng.normal(0, 1, (B, n_out)).astype(np.float32)
    dx, dt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = m.forward(dx).cpu().numpy()
    p = gpu_params_for_reference(m, n_in, width, depth, n_out)
    y_ref = M.forward(p, x, n_in, width, depth, n_out)
    assert np.abs(y - y_ref).max() <= 2e-2 * np.abs(y_ref).max()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    mask = np.where(rng.random((B, n_out)) < 0.7, rng.uniform(0.05, 2.0, (B, n_out)), 0.0).astype(np.float32)
    m.backward(dx, dt, loss, mask=torch.from_numpy(mask).cuda())
    torch.cuda.synchronize()
    g = m.get(1).astype(np.float64)
    l_ref, g_ref = M.loss_and_grad(p, x, t, n_in, width, depth, n_out, mask=mask)
    assert abs(loss.item() - l_ref) <= 1e-2 * l_ref
    lay, _ = M.layout(n_in, width, depth, n_out)
    for (wo, bo, fo, fi) in lay:
        for a, b in ((wo, wo + fo * fi), (bo, bo + fo)):
            gg, gr = g[a:b], g_ref[a:b]
            rel = np.linalg.norm(gg - gr) / np.linalg.norm(gr)
            cos = gg @ gr / (np.linalg.norm(gg) * np.linalg.norm(gr))
            assert rel < 3e-2 and cos > 0.999, (a, rel, cos)
    m.close()


def test_gradients_elementwise_at_the_product_shape():
    """The surrogate's own shape (62 features -> 3 x 256 -> 2048 outputs, batch 1024, so the
    weight-gradient GEMMs take the split-K path): every gradient element against the FP64
    reference with the GPU's BF16-rounded weights. The GEMM operands of layers >= 1 are BF16
    (relative rounding <= 2^-9 each) with FP32 accumulation, so each element's error is at most
    about 2 x 2^-9 times the sum of the magnitudes of the products it adds up
    (oracle.mlp.grad_magnitudes): one rounding per operand, the rounding carried back through the
    layers and the FP32 sums being far smaller (observed at most 0.58 x 2^-9 times that sum, in the
    last layer's weights)."""
    import torch
    rng = np.random.default_rng(5)
    n_in, width, depth, n_out, B = 62, 256, 3, 2048, 1024
    m = rad.MLP(n_in, width, depth, n_out, max_batch=B, seed=8)
    x = rng.uniform(-1, 1, (B, n_in)).astype(np.float32)
    t = rng.normal(0, 1, (B, n_out)).astype(np.float32)
    mask = np.where(rng.random((B, n_out)) < 0.8, rng.uniform(0.02, 1.0, (B, n_out)), 0.0).astype(np.float32)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    m.backward(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), loss, mask=torch.from_numpy(mask).cuda())
    torch.cuda.synchronize()
    g = m.get(1).astype(np.float64)
    p = gpu_params_for_reference(m, n_in, width, depth, n_out)
    _, g_ref = M.loss_and_grad(p, x, t, n_in, width, depth, n_out, mask=mask)
    mag = M.grad_magnitudes(p, x, t, n_in, width, depth, n_out, mask=mask)
    ratio = np.abs(g - g_ref) / (2.0 ** -9 * mag + 1e-30)
    lay, _ = M.layout(n_in, width, depth, n_out)
    worst = [float(ratio[wo:bo + fo].max()) for (wo, bo, fo, fi) in lay]
    print("max |dg| / (2^-9 sum|products|) per layer:", worst, "p99:", float(np.quantile(ratio, 0.99)))
    assert ratio.max() <= 2.0, worst
    m.close()


@pytest.mark.parametrize("n_in,width,depth,n_out,B", [(5, 130, 2, 206, 300), (64, 8, 3, 2, 129)])
def test_gradients_elementwise_at_ragged_shapes(n_in, width, depth, n_out, B):
    """Shapes that are no multiple of the GEMM's 128 x 128 tile or its 64-wide K step, and leading
    dimensions that are no multiple of 8 (width 130: the operand tiles are staged element by
    element instead of 16 bytes at a time), a batch of 300 for the split-K weight gradients, a
    width of 8 and a two-output layer: every gradient element within the bound of the product
    shape's test."""
    import torch
    rng = np.random.default_rng(9)
    m = rad.MLP(n_in, width, depth, n_out, max_batch=B, seed=4)
    x = rng.uniform(-1, 1, (B, n_in)).astype(np.float32)
    t = rng.normal(0, 1, (B, n_out)).astype(np.float32)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    m.backward(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), loss)
    torch.cuda.synchronize()
    g = m.get(1).astype(np.float64)
    p = gpu_params_for_reference(m, n_in, width, depth, n_out)
    _, g_ref = M.loss_and_grad(p, x, t, n_in, width, depth, n_out)
    mag = M.grad_magnitudes(p, x, t, n_in, width, depth, n_out)
    ratio = np.abs(g - g_ref) / (2.0 ** -9 * mag + 1e-30)
    print("ragged shape", (n_in, width, depth, n_out, B), "max ratio", float(ratio.max()))
    assert ratio.max() <= 2.0
    y = m.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    y_ref = M.forward(p, x, n_in, width, depth, n_out)
    assert np.abs(y - y_ref).max() <= 2e-2 * np.abs(y_ref).max()
    assert rad.rad_device_status(1) == rad.RAD_OK
    m.close()


def test_adamw_matches_reference():
    """Two AdamW steps (moments, bias correction, decoupled weight decay) against the FP64
    reference fed the GPU's own gradients; eps comparable to the gradients so that the update is
    not just their sign."""
    import torch
    rng = np.random.default_rng(6)
    n_in, width, depth, n_out, B = 3, 64, 2, 32, 64
    m = rad.MLP(n_in, width, depth, n_out, max_batch=B, seed=2)
    x = torch.from_numpy(rng.uniform(-1, 1, (B, n_in)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.normal(0, 1, (B, n_out)).astype(np.float32)).cuda()
    lr, b1, b2, wd = 1e-2, 0.8, 0.95, 0.05
    p = m.get(0).astype(np.float64)
    mom, vel = np.zeros_like(p), np.zeros_like(p)
    for step in (1, 2):
        m.backward(x, t)
        g = m.get(1).astype(np.float64)
        eps = float(np.median(np.abs(g)))
        m.adamw(lr, b1, b2, eps, wd)
        torch.cuda.synchronize()
        p, mom, vel = M.adamw_step(p, g, mom, vel, step, lr, b1, b2, eps, wd)
        np.testing.assert_allclose(m.get(2), mom, rtol=1e-5, atol=1e-7 * np.abs(mom).max())
        np.testing.assert_allclose(m.get(3), vel, rtol=1e-5, atol=1e-7 * np.abs(vel).max())
        np.testing.assert_allclose(m.get(0), p, rtol=0, atol=2e-6 * (1 + np.abs(p)).max())
    m.close()


def test_training_reduces_loss():
    import torch
    rng = np.random.default_rng(2)
    n_in, n_out, B = 3, 128, 256
    m = rad.MLP(n_in, 128, 3, n_out, max_batch=B, seed=4)
    x = rng.uniform(-1, 1, (B, n_in)).astype(np.float32)
    A = rng.normal(0, 1.5, (n_in, n_out))
    t = np.sin(x @ A).astype(np.float32)
    dx, dt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    m.backward(dx, dt, loss)
    first = loss.item()
    for _ in range(400):
        m.train_step(dx, dt, 3e-3, 0.0, loss)
    assert loss.item() < first / 10
    # parameters round-trip through host memory (checkpoint)
    p = m.get(0)
    m2 = rad.MLP(n_in, 128, 3, n_out, max_batch=B, seed=9)
    m2.set_params(p)
    assert torch.equal(m.forward(dx), m2.forward(dx))
    m.close()
    m2.close()


def test_label_and_ensemble_kernels():
    import torch
    rng = np.random.default_rng(3)
    v = rng.lognormal(0, 3, (50, 40))
    v[0, 0] = 0.0
    dv = torch.from_numpy(v).cuda()
    y = torch.empty(v.shape, dtype=torch.float32, device="cuda")
    rad.rad_log_targets(dv.view(-1), 1e-3, y.view(-1))
    np.testing.assert_allclose(y.cpu().numpy(), np.log10(np.maximum(v, 1e-3)), rtol=1e-6, atol=1e-6)
    mean = torch.empty(40, dtype=torch.float32, device="cuda")
    std = torch.empty(40, dtype=torch.float32, device="cuda")
    rad.rad_column_stats(y, mean, std)
    yn = y.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(mean.cpu().numpy(), yn.mean(0), rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(std.cpu().numpy(), yn.std(0, ddof=1), rtol=1e-5)
    y0 = y.clone()
    rad.rad_standardize(y, mean, std)
    rad.rad_standardize(y, mean, std, inverse=True)
    np.testing.assert_allclose(y.cpu().numpy(), y0.cpu().numpy(), rtol=1e-5, atol=1e-5)
    preds = rng.normal(0, 0.01, (3, 20, 30)).astype(np.float32)
    dp = torch.from_numpy(preds).cuda()
    mu = torch.empty((20, 30), dtype=torch.float32, device="cuda")
    err = torch.empty(20, dtype=torch.float32, device="cuda")
    rad.rad_mlp_ensemble_estimate(dp, mu, err)
    np.testing.assert_allclose(mu.cpu().numpy(), preds.mean(0), rtol=1e-5, atol=1e-7)
    p64 = preds.astype(np.float64)
    p64 = (p64 + np.linspace(-3, 0, 30)[None, None, :]).astype(np.float32).astype(np.float64)  # three decades
    dp.copy_(torch.from_numpy(p64.astype(np.float32)))
    rad.rad_mlp_ensemble_estimate(dp, mu, err)
    s2 = 10.0 ** (2 * p64.mean(0))
    ref = np.log(10) * np.sqrt((s2 * p64.var(0, ddof=1)).sum(1) / s2.sum(1))
    np.testing.assert_allclose(err.cpu().numpy(), ref, rtol=1e-4)
