"""FP64 oracle of the comparison renderer: the indenter's depth map smoothed
by a Gaussian kernel and shaded with the Phong model.

TEST INFRASTRUCTURE ONLY (imported by ``tests/``; the product never imports
it).

Sec. II of the paper describes the simulators Tacchi is measured against:
they build a pseudo elastomer surface by smoothing the indenter's depth map
with Gaussian kernels, with no physics, and shade it the same way (Sec.
III-B follows their shading).  Readings (the paper gives no formula):
  * depth map: per pixel centre (x, y) the penetration p = max(0, z_top -
    z_b(x, y)) of the indenter's lowest point z_b into the rest top face;
  * smoothing: s = sum_{|k|<=Rx, |l|<=Ry} g_x(k) g_y(l) p(x + k PW, y + l PH),
    g(k) proportional to exp(-(k P)^2 / (2 sigma^2)), normalised over
    |k| <= R = ceil(3 sigma / P); p beyond the window comes from the shape;
  * surface: H = z_top - s, shaded by Eqs. 12-14 (the oracle's `shade`).
Pinned in tests/test_oracle_smoothed_pins.py (volumes and footprints of the
shapes in closed form, a height map sampled from a sphere, the discrete
Gaussian of scipy.ndimage, conservation of the pressed volume).

Shapes (the indenter kinds of the library, in the local frame of the pose;
yaw about the vertical only):
  sphere (R): lowest point c_z - sqrt(R^2 - r^2) for r < R;
  cylinder (R, L) along local x: c_z - sqrt(R^2 - y_l^2), |x_l| <= L, |y_l| < R;
  cone (half angle t, height Hc), apex at the pose: c_z + r / tan t for r <= Hc tan t;
  prism (half angle t, half length L along y, height Hp), edge at the pose:
    c_z + |x_l| / tan t for |y_l| <= L, |x_l| <= Hp tan t;
  height map (protrusions hm >= 0 below the back plane, pixel spacing hp,
    row j along local y, sample centres at ((i - (W-1)/2) hp, (j - (H-1)/2) hp)):
    c_z - bilinear(hm) inside the map's extent (clamped to the edge samples).
"""
from __future__ import annotations

import math

import numpy as np

SPHERE, CYLINDER, CONE, PRISM, HEIGHTMAP = 1, 2, 3, 4, 5


def yaw_of(pose):
    qw, qx, qy, qz = pose[3:7]
    n = math.sqrt(qw * qw + qx * qx + qy * qy + qz * qz)
    if abs(qx) > 1e-9 * n or abs(qy) > 1e-9 * n:
        raise ValueError("only rotations about the vertical axis")
    return 2.0 * math.atan2(qz, qw)


def indenter_bottom(kind, params, pose, X, Y, hm=None, hm_pixel=None):
    """Lowest point (m) of the indenter over world points (X, Y); +inf where
    the shape is absent."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    yaw = yaw_of(pose)
    cx, cy, cz = pose[0], pose[1], pose[2]
    dx, dy = X - cx, Y - cy
    lx = math.cos(yaw) * dx + math.sin(yaw) * dy
    ly = -math.sin(yaw) * dx + math.cos(yaw) * dy
    inf = np.inf
    if kind == SPHERE:
        R = params[0]
        r2 = lx * lx + ly * ly
        return np.where(r2 < R * R, cz - np.sqrt(np.maximum(R * R - r2, 0.0)), inf)
    if kind == CYLINDER:
        R, L = params[0], params[1]
        ok = (np.abs(lx) <= L) & (np.abs(ly) < R)
        return np.where(ok, cz - np.sqrt(np.maximum(R * R - ly * ly, 0.0)), inf)
    if kind == CONE:
        t = math.tan(params[0])
        r = np.hypot(lx, ly)
        return np.where(r <= params[1] * t, cz + r / t, inf)
    if kind == PRISM:
        t = math.tan(params[0])
        ok = (np.abs(ly) <= params[1]) & (np.abs(lx) <= params[2] * t)
        return np.where(ok, cz + np.abs(lx) / t, inf)
    if kind == HEIGHTMAP:
        hm = np.asarray(hm, np.float64)
        Hh, Ww = hm.shape
        fx = lx / hm_pixel + (Ww - 1) / 2.0
        fy = ly / hm_pixel + (Hh - 1) / 2.0
        inside = (fx >= -0.5) & (fx <= Ww - 0.5) & (fy >= -0.5) & (fy <= Hh - 0.5)
        fx = np.clip(fx, 0.0, Ww - 1.0)
        fy = np.clip(fy, 0.0, Hh - 1.0)
        ix = np.minimum(np.floor(fx).astype(np.int64), Ww - 2)
        iy = np.minimum(np.floor(fy).astype(np.int64), Hh - 2)
        tx, ty = fx - ix, fy - iy
        h = (hm[iy, ix] * (1 - tx) * (1 - ty) + hm[iy, ix + 1] * tx * (1 - ty)
             + hm[iy + 1, ix] * (1 - tx) * ty + hm[iy + 1, ix + 1] * tx * ty)
        return np.where(inside, cz - h, inf)
    raise ValueError(f"indenter kind {kind}")


def penetration(kind, params, pose, X, Y, z_top, hm=None, hm_pixel=None):
    """p = max(0, z_top - z_b(X, Y)) (m)."""
    zb = indenter_bottom(kind, params, pose, X, Y, hm, hm_pixel)
    return np.maximum(z_top - zb, 0.0)


def radius(sigma_m, pitch_m):
    """Half width (pixels) of the truncated kernel: ceil(3 sigma / P)."""
    return int(math.ceil(3.0 * sigma_m / pitch_m)) if sigma_m > 0 else 0


def gaussian_weights(sigma_m, pitch_m):
    """Normalised discrete Gaussian g[-R..R] on a pixel lattice of pitch P."""
    R = radius(sigma_m, pitch_m)
    if R == 0:
        return np.ones(1)
    k = np.arange(-R, R + 1, dtype=np.float64)
    g = np.exp(-(k * pitch_m) ** 2 / (2.0 * sigma_m ** 2))
    return g / g.sum()


def pixel_lattice(window, w, h, rx=0, ry=0):
    """Pixel-centre coordinates of the window extended by rx, ry pixels."""
    PW = (window[2] - window[0]) / w
    PH = (window[3] - window[1]) / h
    xs = window[0] + (np.arange(-rx, w + rx) + 0.5) * PW
    ys = window[1] + (np.arange(-ry, h + ry) + 0.5) * PH
    return xs, ys, PW, PH


def smooth(p_ext, gx, gy):
    """Direct 2D sum of the product kernel over the extended map p_ext
    [h + 2Ry][w + 2Rx]; returns the [h][w] interior."""
    Ry, Rx = len(gy) // 2, len(gx) // 2
    h, w = p_ext.shape[0] - 2 * Ry, p_ext.shape[1] - 2 * Rx
    s = np.zeros((h, w))
    for l in range(-Ry, Ry + 1):
        for k in range(-Rx, Rx + 1):
            s += gy[l + Ry] * gx[k + Rx] * p_ext[Ry + l:Ry + l + h, Rx + k:Rx + k + w]
    return s


def smoothed_height(kind, params, pose, z_top, window, w, h, sigma_m, hm=None, hm_pixel=None):
    """H = z_top - (Gaussian-smoothed penetration) over the window's pixels."""
    PW = (window[2] - window[0]) / w
    PH = (window[3] - window[1]) / h
    gx, gy = gaussian_weights(sigma_m, PW), gaussian_weights(sigma_m, PH)
    xs, ys, _, _ = pixel_lattice(window, w, h, len(gx) // 2, len(gy) // 2)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    p = penetration(kind, params, pose, X, Y, z_top, hm, hm_pixel)
    return z_top - smooth(p, gx, gy)


def render_smoothed(kind, params, pose, z_top, window, w, h, sigma_m, rp, hm=None, hm_pixel=None):
    """(H, image) of the comparison renderer; shading by the oracle's Eqs. 12-14."""
    from . import shade
    H = smoothed_height(kind, params, pose, z_top, window, w, h, sigma_m, hm, hm_pixel)
    PW = (window[2] - window[0]) / w
    PH = (window[3] - window[1]) / h
    return H, shade(H, PW, PH, z_top, rp)
