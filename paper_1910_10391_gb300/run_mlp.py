"""Time the surrogate network's kernels (rad_mlp_*): training steps and inference.

  python -m paper_1910_10391_gb300.run_mlp --batch 1024 --steps 200

The network is the surrogate's (3 inputs -> 3 hidden layers of 256, GELU -> 2048 outputs; the
first layer FP32, the others BF16 tensor-core GEMMs with FP32 accumulation). Prints one JSON line
with the CUDA-event time per training step (forward, backward, AdamW) and per forward pass, and
the GEMM FLOP rate they imply (2 m n k per GEMM: forward 1, backward 2 GEMMs per BF16 layer).
"""
from __future__ import annotations

import argparse
import json

from . import _binding as rad


def gemm_flops(batch: int, n_in: int, width: int, depth: int, n_out: int) -> tuple:
    """FLOPs of the BF16 GEMMs of one forward pass and of one training step."""
    dims = [width] * depth + [n_out]
    fwd = sum(2.0 * batch * dims[i] * dims[i + 1] for i in range(len(dims) - 1))
    # backward: the input gradient and the weight gradient of every BF16 layer (the input
    # gradient of the first one feeds the FP32 first layer), two GEMMs of the forward's size
    return fwd, 3.0 * fwd


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--width", type=int, default=256)
    ap.add_argument("--depth", type=int, default=3)
    ap.add_argument("--n-out", type=int, default=2048)
    ap.add_argument("--steps", type=int, default=200)
    a = ap.parse_args(argv)
    import torch
    torch.manual_seed(0)
    net = rad.MLP(3, a.width, a.depth, a.n_out, max_batch=a.batch, seed=1)
    x = torch.rand(a.batch, 3, device="cuda")
    t = torch.randn(a.batch, a.n_out, device="cuda") * 0.1
    y = torch.empty(a.batch, a.n_out, device="cuda")
    loss = torch.zeros(1, device="cuda")
    st = torch.cuda.current_stream()

    def timed(fn, n):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(n):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    ms_train = timed(lambda: net.train_step(x, t, 1e-4, 0.0, loss), a.steps)
    ms_fwd = timed(lambda: net.forward(x, y), a.steps)
    status = rad.rad_device_status(1)
    if status:
        raise rad.RadError(status, "device status")
    f_fwd, f_train = gemm_flops(a.batch, 3, a.width, a.depth, a.n_out)
    print(json.dumps({"batch": a.batch, "width": a.width, "depth": a.depth, "n_out": a.n_out,
                      "params": net.num_params, "ms_train_step": ms_train, "ms_forward": ms_fwd,
                      "train_steps_per_s": 1e3 / ms_train, "samples_per_s_inference": a.batch * 1e3 / ms_fwd,
                      "gemm_tflops_train": f_train / (ms_train * 1e-3) / 1e12,
                      "gemm_tflops_forward": f_fwd / (ms_fwd * 1e-3) / 1e12,
                      "loss": float(loss.item())}))
    net.close()


if __name__ == "__main__":
    main()
