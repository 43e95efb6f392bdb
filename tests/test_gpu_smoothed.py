"""Comparison renderer (the Gaussian depth-smoothing simulators of Sec. II)
against the FP64 oracle: the smoothed height map and its shading for every
indenter kind, with a yaw, a window that cuts through the contact (the
penetration beyond the window comes from the shape), non-square pixels,
sigma = 0, host output buffers and the argument checks.

Tolerances: the GPU evaluates the shapes in FP32 at metre scale (z ~ 5e-3 m,
ulp 4.7e-10 m), so the height map agrees to 5 nm; the shading (central
differences over 0.1 mm pixels, then Eqs. 12-14 in FP32) to 1e-4."""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def T():
    import paper_2301_08343_gb300 as P
    return P


def oracle_rp():
    import oracle
    Lt = W.default_lights()
    return oracle.render_params(Lt["n_lights"], Lt["dirs"], Lt["diffuse"], Lt["specular"], Lt["ambient"],
                                Lt["ka"], Lt["kd"], Lt["ks"], Lt["alpha"])


def tapered_hm():
    hm = np.asarray(W.hm_perlin(n=40, pix=0.15e-3, seed=5, amp=0.8e-3), np.float64)
    t = np.sin(np.linspace(0, math.pi, 40)) ** 2
    return (hm * t[:, None] * t[None, :]).astype(np.float32)


CASES = {
    "sphere": (1, (3e-3,), 3e-3 - 0.6e-3),
    "cylinder": (2, (1.5e-3, 4e-3), 1.5e-3 - 0.5e-3),
    "cone": (3, (math.radians(35), 3e-3), -0.5e-3),
    "prism": (4, (math.radians(45), 4e-3, 3e-3), -0.4e-3),
    "heightmap": (5, (1.5e-3,), 0.1e-3),
}


@pytest.mark.parametrize("kind", list(CASES))
@pytest.mark.parametrize("sigma", [0.0, 0.25e-3, 0.6e-3])
def test_smoothed_render_matches_oracle(kind, sigma):
    from oracle import smoothed as S
    P = T()
    b = W.C3_BLOCK
    bt = P.TacchiBatch([b])
    z_top = b.nz * b.dx
    k, params, lift = CASES[kind]
    hm = tapered_hm() if kind == "heightmap" else None
    yaw = 0.7
    c = (6.3e-3, 5.8e-3, z_top + lift)
    pose = c + (math.cos(yaw / 2), 0.0, 0.0, math.sin(yaw / 2))
    bt.set_indenter(0, k, params, pose, (0,) * 6, hm=hm, hm_pixel=0.15e-3)
    # a window that cuts through the contact, with non-square pixels
    win = (5.5e-3, 2.0e-3, 12.7e-3, 9.6e-3)
    w, h = 96, 64
    Hd = torch.empty((h, w), device="cuda")
    img = bt.render_smoothed(0, w, h, win, sigma, rp=P.render_params_from(W.default_lights()), out_height=Hd)
    Hg = Hd.cpu().numpy().astype(np.float64)
    Ho, Io = S.render_smoothed(k, params, pose, z_top, win, w, h, sigma, oracle_rp(),
                               None if hm is None else hm.astype(np.float64), 0.15e-3)
    assert (z_top - Ho).max() > 1e-5  # the contact is in the window
    assert np.abs(Hg - Ho).max() <= 5e-9
    assert np.abs(img.cpu().numpy() - Io).max() <= 1e-4


def test_host_buffers_zero_sigma_is_the_penetration_map_and_checks():
    import ctypes as C
    from paper_2301_08343_gb300 import _lib
    P = T()
    b = W.C3_BLOCK
    bt = P.TacchiBatch([b])
    z_top = b.nz * b.dx
    bt.set_indenter(0, P.IndenterKind.SPHERE, (3e-3,), (6e-3, 6e-3, z_top + 2.5e-3, 1, 0, 0, 0), (0,) * 6)
    win = W.top_window(b)
    Hd = torch.empty((48, 48), device="cuda")
    dev = bt.render_smoothed(0, 48, 48, win, 0.3e-3, out_height=Hd)
    host = np.zeros((48, 48, 3), np.float32)
    hh = np.zeros((48, 48), np.float32)
    st = _lib.lib().tacchi_batch_render_smoothed(bt._h, 0, C.byref(P.default_render_params()), 48, 48,
                                                 (C.c_double * 4)(*win), 0.3e-3, _lib.ptr(host), _lib.ptr(hh))
    assert st == 0
    assert np.array_equal(host, dev.cpu().numpy()) and np.array_equal(hh, Hd.cpu().numpy())
    bt.render_smoothed(0, 48, 48, win, 0.0, out_height=Hd)
    pen = bt.penetration_map(0, 48, 48, win)
    assert torch.allclose(Hd, z_top - pen, rtol=0, atol=1e-9)
    # sigma so large that the kernel would exceed 256 pixels; a negative sigma
    with pytest.raises(RuntimeError):
        bt.render_smoothed(0, 48, 48, win, 100 * (win[2] / 48), out_height=Hd)
    with pytest.raises(RuntimeError):
        bt.render_smoothed(0, 48, 48, win, -1e-4, out_height=Hd)
    assert bt.status() == 0


def test_full_frame_sampled_pixels():
    """The 640 x 480 frame of the A/B benchmark (the 12 x 12 mm top face,
    sigma 0.7 mm: kernels of 112 x 84 pixels half width): sampled pixels
    against the oracle's direct sum over each pixel's own kernel footprint."""
    from oracle import smoothed as S
    P = T()
    b = W.C3_BLOCK
    bt = P.TacchiBatch([b])
    z_top = b.nz * b.dx
    R, d, yaw = 3e-3, 0.8e-3, 0.4
    pose = (6.4e-3, 5.7e-3, z_top + R - d, math.cos(yaw / 2), 0.0, 0.0, math.sin(yaw / 2))
    bt.set_indenter(0, P.IndenterKind.CYLINDER, (R, 4e-3), pose, (0,) * 6)
    win = W.top_window(b)
    w, h, sigma = 640, 480, 0.7e-3
    Hd = torch.empty((h, w), device="cuda")
    bt.render_smoothed(0, w, h, win, sigma, out_height=Hd)
    Hg = Hd.cpu().numpy().astype(np.float64)
    gx = S.gaussian_weights(sigma, (win[2] - win[0]) / w)
    gy = S.gaussian_weights(sigma, (win[3] - win[1]) / h)
    rx, ry = len(gx) // 2, len(gy) // 2
    assert (rx, ry) == (112, 84)
    xs, ys, _, _ = S.pixel_lattice(win, w, h, rx, ry)
    rng = np.random.default_rng(2)
    pix = [(h // 2, w // 2), (0, 0), (h - 1, w - 1)] + [tuple(q) for q in
                                                        rng.integers((0, 0), (h, w), size=(150, 2))]
    worst = 0.0
    for r, c in pix:
        X, Y = np.meshgrid(xs[c:c + 2 * rx + 1], ys[r:r + 2 * ry + 1], indexing="xy")
        p = S.penetration(S.CYLINDER, (R, 4e-3), pose, X, Y, z_top)
        s = S.smooth(p, gx, gy)[0, 0]
        worst = max(worst, abs(Hg[r, c] - (z_top - s)))
    assert float((z_top - Hd).max()) > 0.3e-3
    assert worst <= 5e-9, worst
