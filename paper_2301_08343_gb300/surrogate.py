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


def per_frame_rms_um(pred, Y):
    """RMS of the vertical displacement error of every frame (um), numpy."""
    import torch
    dz = (pred[..., 2] - Y[..., 2]) * 1e3
    return torch.sqrt((dz ** 2).mean(dim=(1, 2))).cpu().numpy()


def depth_bin(depth_m, width_m=0.1e-3):
    return int(depth_m / width_m + 1e-9)


def calibrate_region(rms_um, specs, gate_um=5.0, width_m=0.1e-3, min_frames=8):
    """The validity region of a trained surrogate: the (shape, depth bin)
    cells whose held-out frames all meet the gate at the 99th percentile of
    their per-frame RMS error (cells with fewer than min_frames frames are
    left out).  Returns a sorted list of (kind, bin) pairs."""
    groups = {}
    for e, sp in zip(rms_um, specs):
        groups.setdefault((sp["kind"], depth_bin(sp["depth"], width_m)), []).append(float(e))
    return sorted(k for k, v in groups.items() if len(v) >= min_frames and np.percentile(v, 99) <= gate_um)


def in_region(region, kind, depth_m, width_m=0.1e-3):
    return (kind, depth_bin(depth_m, width_m)) in set(map(tuple, region))


def errors_by_group(rms_um, specs, width_m=0.1e-3):
    """Per shape and per depth bin: frames, mean and p99 of the per-frame RMS
    error (um)."""
    out = {}
    for key_of in (lambda sp: sp["kind"], lambda sp: f"{depth_bin(sp['depth'], width_m) * width_m * 1e3:.1f}mm"):
        groups = {}
        for e, sp in zip(rms_um, specs):
            groups.setdefault(key_of(sp), []).append(float(e))
        for k, v in sorted(groups.items()):
            out[k] = {"n": len(v), "mean": float(np.mean(v)), "p99": float(np.percentile(v, 99))}
    return out


def tactile_images(uz_mm, block, rp=None):
    """Tactile images (Sec. III-B, Eqs. 12-14) of vertical top-surface
    displacement maps uz_mm [n, h, w] (mm, over the block's top face): the
    height map H = z_top + u_z shaded by the library's kernel.  Returns
    [n, h, w, 3] on the device."""
    import torch
    from . import default_render_params, shade
    rp = rp or default_render_params()
    n, h, w = uz_mm.shape
    z_top = block.nz * block.dx
    out = torch.empty((n, h, w, 3), device=uz_mm.device)
    H = (z_top + uz_mm * MM).float().contiguous()
    for i in range(n):
        shade(H[i], block.nx * block.dx / w, block.ny * block.dx / h, z_top, rp, out=out[i])
    return out


def image_errors(img, ref):
    """Per-frame RMS difference of two tactile image stacks (intensity in
    [0, 1], over pixels and channels): mean, p99, max, and the mean PSNR."""
    import torch
    rms = torch.sqrt(((img - ref) ** 2).mean(dim=(1, 2, 3))).cpu().numpy()
    psnr = -20.0 * np.log10(np.maximum(rms, 1e-12))
    return {"rms_mean": float(rms.mean()), "rms_p99": float(np.percentile(rms, 99)), "rms_max": float(rms.max()),
            "psnr_db_mean": float(psnr.mean())}


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
