"""FP64 numpy oracle of the learned surrogate network (forward, analytic
backward, Adam).

TEST INFRASTRUCTURE ONLY (tests/ and bench.py's baseline leg).  The paper has
no surrogate; this oracle follows the network the library trains:

  U-Net on NHWC images.  Encoder levels l = 0..L-1 with widths c_l: two 3x3
  'same' convolutions with bias and ReLU, then (except the last level) 2x2
  average pooling.  Decoder levels l = L-2..0: nearest-neighbour 2x
  upsampling, channel concatenation [upsampled, skip], two 3x3 conv+ReLU.
  Head: 1x1 convolution to the output channels, no activation.  Loss: mean
  of squared errors over all outputs.

Parameters are a dict name -> array; 3x3 weights are [3, 3, C_in, C_out]
(tap y, tap x, input channel, output channel), 1x1 head [C_in, C_out].
Convolution is cross-correlation: out[y, x, o] = b[o] + sum_{dy, dx, i}
W[dy, dx, i, o] * in[y + dy - 1, x + dx - 1, i], zero outside the image.
"""
from __future__ import annotations

import numpy as np


def conv3x3(x, W, b):
    """x [N, H, W, Ci] -> [N, H, W, Co]; plain sum over the nine taps."""
    n, h, w, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((n, h, w, W.shape[3]))
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("nhwi,io->nhwo", xp[:, dy:dy + h, dx:dx + w, :], W[dy, dx])
    return out + b


def conv3x3_backward(x, W, gout):
    """Gradients of conv3x3 with respect to x, W and b."""
    n, h, w, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    gW = np.zeros_like(W)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            gW[dy, dx] = np.einsum("nhwi,nhwo->io", xp[:, dy:dy + h, dx:dx + w, :], gout)
            gxp[:, dy:dy + h, dx:dx + w, :] += np.einsum("nhwo,io->nhwi", gout, W[dy, dx])
    gb = gout.sum(axis=(0, 1, 2))
    return gxp[:, 1:-1, 1:-1, :], gW, gb


def avgpool2(x):
    n, h, w, c = x.shape
    return x.reshape(n, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))


def avgpool2_backward(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_backward(g):
    n, h, w, c = g.shape
    return g.reshape(n, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


def layer_names(widths):
    """Conv layers in execution order: (name, C_in, C_out)."""
    L = len(widths)
    names = []
    for l in range(L):
        cin = widths[l - 1] if l > 0 else None
        names.append((f"enc{l}a", cin, widths[l]))
        names.append((f"enc{l}b", widths[l], widths[l]))
    for l in range(L - 2, -1, -1):
        names.append((f"dec{l}a", widths[l + 1] + widths[l], widths[l]))
        names.append((f"dec{l}b", widths[l], widths[l]))
    return names


def init_params(widths, c_in, c_out, seed):
    """He-normal 3x3 weights, zero biases (numpy PCG64 seeded)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, ci, co in layer_names(widths):
        ci = c_in if ci is None else ci
        P[name + ".W"] = rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), (3, 3, ci, co))
        P[name + ".b"] = np.zeros(co)
    P["head.W"] = rng.normal(0.0, np.sqrt(1.0 / widths[0]), (widths[0], c_out))
    P["head.b"] = np.zeros(c_out)
    return P


def forward(P, x, widths):
    """Returns the output and the cache needed by backward."""
    L = len(widths)
    cache = {}
    skips = []
    h = x
    for l in range(L):
        for s in "ab":
            name = f"enc{l}{s}"
            cache[name + ".in"] = h
            h = np.maximum(conv3x3(h, P[name + ".W"], P[name + ".b"]), 0.0)
            cache[name + ".out"] = h
        if l < L - 1:
            skips.append(h)
            h = avgpool2(h)
    for l in range(L - 2, -1, -1):
        h = np.concatenate([upsample2(h), skips[l]], axis=-1)
        for s in "ab":
            name = f"dec{l}{s}"
            cache[name + ".in"] = h
            h = np.maximum(conv3x3(h, P[name + ".W"], P[name + ".b"]), 0.0)
            cache[name + ".out"] = h
    cache["head.in"] = h
    y = np.einsum("nhwi,io->nhwo", h, P["head.W"]) + P["head.b"]
    return y, cache


def loss_and_grad(P, x, target, widths):
    """Mean squared error and its gradient with respect to every parameter."""
    L = len(widths)
    y, cache = forward(P, x, widths)
    diff = y - target
    loss = float(np.mean(diff ** 2))
    gy = 2.0 * diff / diff.size
    G = {}
    h = cache["head.in"]
    G["head.W"] = np.einsum("nhwi,nhwo->io", h, gy)
    G["head.b"] = gy.sum(axis=(0, 1, 2))
    g = np.einsum("nhwo,io->nhwi", gy, P["head.W"])
    skip_grads = [None] * L
    # decoder in reverse execution order: level 0 first, then up to L-2
    for l in range(0, L - 1):
        for s in "ba":
            name = f"dec{l}{s}"
            g = g * (cache[name + ".out"] > 0)
            g, G[name + ".W"], G[name + ".b"] = conv3x3_backward(cache[name + ".in"], P[name + ".W"], g)
        cu = widths[l + 1]
        skip_grads[l] = g[..., cu:]
        g = upsample2_backward(g[..., :cu])  # gradient of the level l+1 output
    # encoder in reverse execution order
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            g = avgpool2_backward(g) + skip_grads[l]
        for s in "ba":
            name = f"enc{l}{s}"
            g = g * (cache[name + ".out"] > 0)
            g, G[name + ".W"], G[name + ".b"] = conv3x3_backward(cache[name + ".in"], P[name + ".W"], g)
    return loss, G


def adam(P, G, M, V, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) in place; t counts from 1."""
    for k in P:
        M[k] = b1 * M[k] + (1 - b1) * G[k]
        V[k] = b2 * V[k] + (1 - b2) * G[k] ** 2
        mh = M[k] / (1 - b1 ** t)
        vh = V[k] / (1 - b2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
