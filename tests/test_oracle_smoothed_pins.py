"""Pins of the comparison renderer's oracle (the Gaussian-smoothed indenter
depth map of the simulators in Sec. II) against closed forms and a library
routine:
  * pressed volume of each shape = the closed-form volume of the part below
    the rest face (spherical cap, circular cone, cylinder segment, wedge);
  * the sphere's footprint is the disc of radius sqrt(2 R d - d^2);
  * a height map sampled from a sphere reproduces the sphere at its samples
    (pins the sample layout, the row/column order and the yaw);
  * the discrete Gaussian equals scipy.ndimage.gaussian_filter's, and
    smoothing keeps the pressed volume, keeps a constant field, and is the
    identity at sigma = 0.
"""
import math

import numpy as np
import pytest

from oracle import smoothed as S

Z = 4e-3


def grid(half, n, c=(0.0, 0.0)):
    xs = c[0] + (np.arange(n) + 0.5) * (2 * half / n) - half
    ys = c[1] + (np.arange(n) + 0.5) * (2 * half / n) - half
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    return X, Y, (2 * half / n) ** 2


def yaw_pose(c, yaw):
    return (c[0], c[1], c[2], math.cos(yaw / 2), 0.0, 0.0, math.sin(yaw / 2))


@pytest.mark.parametrize("yaw", [0.0, 0.9])
def test_pressed_volumes_in_closed_form(yaw):
    d = 0.5e-3
    X, Y, dA = grid(4e-3, 2400, (1e-3, -0.5e-3))
    # sphere: cap of height d
    R = 3e-3
    p = S.penetration(S.SPHERE, (R,), yaw_pose((1e-3, -0.5e-3, Z + R - d), yaw), X, Y, Z)
    assert p.sum() * dA == pytest.approx(math.pi * d * d * (3 * R - d) / 3, rel=2e-4)
    # cone of half angle t: a cone of height d and base radius d tan t
    t = math.radians(35)
    p = S.penetration(S.CONE, (t, 3e-3), yaw_pose((1e-3, -0.5e-3, Z - d), yaw), X, Y, Z)
    assert p.sum() * dA == pytest.approx(math.pi * (d * math.tan(t)) ** 2 * d / 3, rel=2e-3)
    # cylinder of radius R and length 2L: circular segment x 2L
    R, L = 1.5e-3, 2e-3
    p = S.penetration(S.CYLINDER, (R, L), yaw_pose((1e-3, -0.5e-3, Z + R - d), yaw), X, Y, Z)
    seg = R * R * math.acos((R - d) / R) - (R - d) * math.sqrt(2 * R * d - d * d)
    assert p.sum() * dA == pytest.approx(seg * 2 * L, rel=2e-3)
    # prism: triangle of depth d and half width d tan t, length 2L
    t, L = math.radians(40), 2.5e-3
    p = S.penetration(S.PRISM, (t, L, 3e-3), yaw_pose((1e-3, -0.5e-3, Z - d), yaw), X, Y, Z)
    assert p.sum() * dA == pytest.approx(d * d * math.tan(t) * 2 * L, rel=2e-3)


def test_sphere_footprint_and_depth():
    R, d = 3e-3, 0.4e-3
    X, Y, dA = grid(3e-3, 600)
    p = S.penetration(S.SPHERE, (R,), (0.0, 0.0, Z + R - d, 1.0, 0.0, 0.0, 0.0), X, Y, Z)
    a = math.sqrt(2 * R * d - d * d)
    r = np.hypot(X, Y)
    pitch = math.sqrt(dA)
    assert np.all(p[r < a - pitch] > 0) and np.all(p[r > a + pitch] == 0)
    assert p.max() == pytest.approx(d, rel=1e-4)


def test_cylinder_yaw_quarter_turn_is_a_transpose():
    X, Y, _ = grid(3e-3, 120)
    pose0 = (0.0, 0.0, Z + 1.5e-3 - 0.3e-3, 1.0, 0.0, 0.0, 0.0)
    p0 = S.penetration(S.CYLINDER, (1.5e-3, 2e-3), pose0, X, Y, Z)
    p1 = S.penetration(S.CYLINDER, (1.5e-3, 2e-3), yaw_pose(pose0[:3], math.pi / 2), X, Y, Z)
    assert np.count_nonzero(p0) > 100
    np.testing.assert_allclose(p1, p0.T, atol=1e-15)


def test_heightmap_sampled_from_a_sphere_reproduces_it():
    R, hp, n = 3e-3, 0.1e-3, 71
    k = (np.arange(n) - (n - 1) / 2) * hp
    lx, ly = np.meshgrid(k, k, indexing="xy")          # row j along local y
    r2 = lx ** 2 + ly ** 2
    hm = np.where(r2 < R * R, np.sqrt(np.maximum(R * R - r2, 0)), 0.0)
    c = (2e-3, 1e-3, Z + R - 0.5e-3)
    yaw = 0.4
    pose = yaw_pose(c, yaw)
    # world positions of the samples
    X = c[0] + math.cos(yaw) * lx - math.sin(yaw) * ly
    Y = c[1] + math.sin(yaw) * lx + math.cos(yaw) * ly
    ph = S.penetration(S.HEIGHTMAP, (1e-3,), pose, X, Y, Z, hm, hp)
    ps = S.penetration(S.SPHERE, (R,), pose, X, Y, Z)
    assert np.count_nonzero(ps) > 500
    np.testing.assert_allclose(ph, ps, atol=1e-15)


def test_gaussian_matches_scipy_and_keeps_volume():
    ndimage = pytest.importorskip("scipy.ndimage")
    win = (0.0, 0.0, 8e-3, 8e-3)
    w = h = 80
    sigma = 0.23e-3
    pose = (4.1e-3, 3.7e-3, Z + 2e-3 - 0.4e-3, 1.0, 0.0, 0.0, 0.0)
    gx = S.gaussian_weights(sigma, 0.1e-3)
    R = len(gx) // 2
    assert R == 7
    xs, ys, PW, PH = S.pixel_lattice(win, w, h, R, R)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    p = S.penetration(S.SPHERE, (2e-3,), pose, X, Y, Z)
    H = S.smoothed_height(S.SPHERE, (2e-3,), pose, Z, win, w, h, sigma)
    sp = sigma / PW
    ref = ndimage.gaussian_filter(p, sp, mode="constant", truncate=R / sp)[R:R + h, R:R + w]
    np.testing.assert_allclose(Z - H, ref, atol=1e-15)
    # the pressed volume is kept (the footprint is well inside the window)
    assert (Z - H).sum() == pytest.approx(p.sum(), rel=1e-12)
    assert (Z - H).max() < p.max()


def test_constant_field_and_zero_sigma():
    win = (0.0, 0.0, 2e-3, 2e-3)
    hm = np.full((8, 8), 0.3e-3)
    pose = (1e-3, 1e-3, Z + 0.1e-3, 1.0, 0.0, 0.0, 0.0)
    H = S.smoothed_height(S.HEIGHTMAP, (1e-3,), pose, Z, win, 20, 20, 0.05e-3, hm, 1e-3)
    np.testing.assert_allclose(H, Z - 0.2e-3, atol=1e-16)
    pose = (1e-3, 0.9e-3, Z + 1e-3 - 0.3e-3, 1.0, 0.0, 0.0, 0.0)
    H0 = S.smoothed_height(S.SPHERE, (1e-3,), pose, Z, win, 20, 20, 0.0)
    xs, ys, _, _ = S.pixel_lattice(win, 20, 20)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    np.testing.assert_array_equal(H0, Z - S.penetration(S.SPHERE, (1e-3,), pose, X, Y, Z))
