"""The surrogate's data path on the GPU: the displacement map (training
target) against a gather written from its definition on the host, the
penetration map (input) against FP64 geometry, and a small end-to-end run of
MPM data generation, training and evaluation showing what the network gains
over running the MPM."""
import math

import numpy as np
import pytest

import oracle
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
    import paper_2301_08343_gb300 as T_
    return T_


def test_displacement_map_is_the_gather_it_defines():
    b = W.Block(10, 8, 3, 0.5e-3, seed=4)
    bt = T().TacchiBatch([W.Block(4, 4, 2, 0.5e-3, seed=1), b])
    u0, fl = oracle.lattice(b.nx, b.ny, b.nz, b.pad_side, b.pad_bottom, b.seed)
    win = (-0.3e-3, 0.2e-3, 5.4e-3, 4.1e-3)
    w, h = 37, 23
    d0 = bt.displacement_map(1, w, h, win).cpu().numpy()
    assert np.all(d0 == 0)
    u, v, Cm, Fm = W.perturbed_state(u0, 9, disp_cells=0.2)
    bt.set_state(1, u, v, Cm, Fm)
    d = bt.displacement_map(1, w, h, win).cpu().numpy()
    # definition: pixel centre -> rest sub-cell (i, j) of the top particle
    # layer -> that particle's displacement
    surf = np.nonzero(fl & 2)[0]
    cx = win[0] + (np.arange(w) + 0.5) * (win[2] - win[0]) / w
    cy = win[1] + (np.arange(h) + 0.5) * (win[3] - win[1]) / h
    for r in range(h):
        for c in range(w):
            i = min(max(int(math.floor(cx[c] / (b.dx / 2))), 0), 2 * b.nx - 1)
            j = min(max(int(math.floor(cy[r] / (b.dx / 2))), 0), 2 * b.ny - 1)
            # the surface particle at lattice (i, j): cell (i//2, j//2) of
            # the top layer, sub-cell (i%2, j%2, 1)
            p = (((b.nz - 1) * b.ny + j // 2) * b.nx + i // 2) * 8 + 4 + (j % 2) * 2 + (i % 2)
            assert p in surf
            exp = (u[:, p].astype(np.float64) - u0[:, p]) * b.dx
            assert np.abs(d[r, c] - exp).max() <= 1e-7 * b.dx


@pytest.mark.parametrize("kind", ["sphere", "cylinder", "cone", "prism"])
def test_penetration_map_matches_fp64_geometry(kind):
    b = W.C3_BLOCK
    bt = T().TacchiBatch([b])
    yaw = 0.7
    z_top = b.nz * b.dx
    K = T().IndenterKind
    params = {"sphere": (3e-3,), "cylinder": (1.5e-3, 4e-3), "cone": (math.radians(35), 3e-3),
              "prism": (math.radians(45), 4e-3, 3e-3)}[kind]
    depth = 0.6e-3
    tip = {"sphere": params[0], "cylinder": params[0], "cone": 0.0, "prism": 0.0}[kind]
    c = (6.3e-3, 5.8e-3, z_top + tip - depth)
    pose = c + (math.cos(yaw / 2), 0.0, 0.0, math.sin(yaw / 2))
    bt.set_indenter(0, getattr(K, kind.upper()), params, pose, (0,) * 6)
    win = W.top_window(b)
    n = 64
    got = bt.penetration_map(0, n, n, win).cpu().numpy()
    xs = win[0] + (np.arange(n) + 0.5) * (win[2] - win[0]) / n
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    dxw, dyw = X - c[0], Y - c[1]
    lx = math.cos(yaw) * dxw + math.sin(yaw) * dyw
    ly = -math.sin(yaw) * dxw + math.cos(yaw) * dyw
    inf = np.inf
    if kind == "sphere":
        r2 = lx ** 2 + ly ** 2
        zb = np.where(r2 < params[0] ** 2, c[2] - np.sqrt(np.maximum(params[0] ** 2 - r2, 0)), inf)
    elif kind == "cylinder":
        zb = np.where((np.abs(lx) <= params[1]) & (np.abs(ly) < params[0]),
                      c[2] - np.sqrt(np.maximum(params[0] ** 2 - ly ** 2, 0)), inf)
    elif kind == "cone":
        r = np.hypot(lx, ly)
        t = math.tan(params[0])
        zb = np.where(r <= params[1] * t, c[2] + r / t, inf)
    else:
        t = math.tan(params[0])
        zb = np.where((np.abs(ly) <= params[1]) & (np.abs(lx) <= params[2] * t), c[2] + np.abs(lx) / t, inf)
    exp = np.maximum(z_top - zb, 0.0)
    assert exp.max() > 0.3e-3  # the tip may fall between pixel centres
    assert np.abs(got - exp).max() <= 2e-8 + 1e-5 * exp.max()


def test_surrogate_learns_the_press_and_beats_mpm_speed():
    from paper_2301_08343_gb300 import surrogate as SG
    specs = W.c3_specs(96, seed_base=7000)
    X, Y, mpm_s = SG.generate(specs, W.C3_BLOCK, W.C3_SUBSTEPS, W.C3_DT, size=64, chunk=96)
    assert torch.isfinite(X).all() and torch.isfinite(Y).all()
    assert float(Y[..., 2].min()) < -0.05  # pressed by tens of micrometres at least
    net = T().SurrogateNet((32, 64, 128, 256), 2, 3, size=64, max_batch=64, seed=3)
    base = SG.errors_um(torch.zeros_like(Y[80:]), Y[80:])
    SG.train(net, X[:80], Y[:80], steps=300, batch=32, lr=2e-3)
    err = SG.errors_um(SG.predict(net, X[80:], batch=16), Y[80:])
    # it has learned most of the vertical displacement on unseen presses
    assert err["rms_uz_um_mean"] < 0.5 * base["rms_uz_um_mean"], (err, base)
    # and one inference frame costs far less than one MPM frame
    mpm_fps = len(specs) / mpm_s
    nn_fps = SG.inference_rate(net, X, batch=64)
    assert nn_fps > 10 * mpm_fps, (nn_fps, mpm_fps)
