"""Learned surrogate of the MPM press (this library's addition; the paper
has none): data generated by the batched MPM, training and evaluation with
the library's BF16 tensor-core network kernels.

Input per sample (64 x 64, over the elastomer's top face): the indenter's
penetration into the rest top face at the end of the press (mm) and the
press depth (mm, constant channel).  Output: the top-surface displacement
(ux, uy, uz in mm) the MPM produces.  Every evaluation reports its error
against held-out MPM results.
"""
from __future__ import annotations

import time

import numpy as np

from . import IndenterKind, SurrogateNet, TacchiBatch

MM = 1.0e-3


def _kind(name):
    return {"sphere": IndenterKind.SPHERE, "cylinder": IndenterKind.CYLINDER,
            "cone": IndenterKind.CONE, "prism": IndenterKind.PRISM}[name]


def generate(specs, block, substeps, dt, size=64, chunk=512, device=None):
    """Run every press of `specs` with the batched MPM (one handle per chunk
    of sensors, each pressed from first contact to its depth over `substeps`
    substeps) and return (X [n,size,size,2], Y [n,size,size,3]) as FP32
    device tensors in mm, plus the MPM time in seconds."""
    import torch
    n = len(specs)
    X = torch.empty((n, size, size, 2), device=device or "cuda")
    Y = torch.empty((n, size, size, 3), device=device or "cuda")
    win = (0.0, 0.0, block.nx * block.dx, block.ny * block.dx)
    mpm_s = 0.0
    for c0 in range(0, n, chunk):
        part = specs[c0:c0 + chunk]
        bt = TacchiBatch([block] * len(part))
        for i, s in enumerate(part):
            bt.set_indenter(i, _kind(s["kind"]), s["params"], s["pose"],
                            (0.0, 0.0, -s["depth"] / (substeps * dt), 0.0, 0.0, 0.0))
        torch.cuda.synchronize()
        t = time.perf_counter()
        bt.step(substeps, dt)
        st = bt.status()
        mpm_s += time.perf_counter() - t
        if st != 0:
            raise RuntimeError(f"MPM data generation failed with status {st}")
        for i, s in enumerate(part):
            X[c0 + i, :, :, 0] = bt.penetration_map(i, size, size, win) / MM
            X[c0 + i, :, :, 1] = s["depth"] / MM
            Y[c0 + i] = bt.displacement_map(i, size, size, win) / MM
        bt.close()
    torch.cuda.synchronize()
    return X, Y, mpm_s


def train(net: SurrogateNet, X, Y, steps, batch=256, lr=1e-3, lr_final=1e-5, seed=0, log_every=0):
    """Adam with cosine-decayed learning rate over random mini-batches."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    losses = []
    for k in range(steps):
        idx = torch.randint(0, n, (batch,), generator=g).to(X.device)
        lr_k = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * k / max(steps - 1, 1)))
        want = log_every and (k % log_every == 0 or k == steps - 1)
        loss = net.train_step(X[idx], Y[idx], lr_k, want_loss=bool(want))
        if want:
            losses.append((k, loss))
    return losses


def predict(net: SurrogateNet, X, batch=1024):
    import torch
    out = torch.empty((X.shape[0], net.size, net.size, net.cout), device=X.device)
    for c0 in range(0, X.shape[0], batch):
        out[c0:c0 + batch] = net.forward(X[c0:c0 + batch])
    return out


def errors_um(pred, Y):
    """Per-sample RMS of the vertical displacement error (um) and its p50,
    p99, max, plus the RMS over all three components."""
    import torch
    dz = (pred[..., 2] - Y[..., 2]) * 1e3  # mm -> um
    rms = torch.sqrt((dz ** 2).mean(dim=(1, 2))).cpu().numpy()
    all_rms = float(torch.sqrt(((pred - Y) * 1e3).pow(2).mean()).item())
    return {"rms_uz_um_mean": float(rms.mean()), "rms_uz_um_p50": float(np.percentile(rms, 50)),
            "rms_uz_um_p99": float(np.percentile(rms, 99)), "max_abs_uz_um": float(dz.abs().max().item()),
            "rms_xyz_um": all_rms, "signal_rms_uz_um": float((Y[..., 2] * 1e3).pow(2).mean().sqrt().item())}


def inference_rate(net: SurrogateNet, X, batch, reps=5):
    """Frames per second of surrogate inference at a batch size."""
    import torch
    x = X[:batch].contiguous()
    out = torch.empty((batch, net.size, net.size, net.cout), device=X.device)
    net.forward(x, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        net.forward(x, out=out)
    e1.record()
    torch.cuda.synchronize()
    return batch * reps / (e0.elapsed_time(e1) * 1e-3)
