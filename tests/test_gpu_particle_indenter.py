"""Indenter represented by particles (the paper's Eq. 10 model) against the
FP64 oracle (GPU, through the C ABI).

Tolerances as for the grid-boundary indenter: one P2G from an identical
state to 1e-5 relative on grid mass and momentum (indenter particles
included, positions rounded to FP32 on the GPU), positions after 200
substeps within 1e-3 cells."""
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
    oracle.set_threads(16)


B = W.Block(10, 9, 3, 0.5e-3, seed=31)
R = 2.0e-3
POSE = (2.5e-3, 2.2e-3, 1.5e-3 + R - 0.1e-3, math.cos(0.15), 0.0, 0.0, math.sin(0.15))
VEL = (0.02, 0.0, -0.25, 0.0, 0.0, 3.0)


def pair(mass=4e-8, n=3000):
    import paper_2301_08343_gb300 as T
    g = T.Tacchi(B.extent_m, B.dx, B.E, B.nu, B.rho, seed=B.seed)
    o = oracle.Sim(B.nx, B.ny, B.nz, B.dx, B.E, B.nu, B.rho)
    u0, fl = oracle.lattice(B.nx, B.ny, B.nz, 4, 3, B.seed, True)
    o.set_state(u0, flags=fl)
    pts = W.indenter_points("sphere", (R,), n, seed=4, reach=0.8e-3).astype(np.float32)
    g.set_indenter(T.IndenterKind.SPHERE, (R,), POSE, VEL)
    g.set_indenter_particles(pts, mass)
    o.set_indenter(oracle.IND_SPHERE, (R,), POSE, VEL)
    o.set_indenter_particles(pts.astype(np.float64), mass)
    return T, g, o, pts


def rel(a, b):
    return np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-300)


def test_grid_of_one_substep_matches_oracle():
    T, g, o, pts = pair()
    g.step(1, 1e-5)
    G = g.get_grid().cpu().numpy().astype(np.float64)
    Mo, MGo = o.p2g(1e-5)
    assert rel(G[:, 0], Mo) <= 1e-5
    assert rel(G[:, 1:].T, MGo) <= 1e-5
    # the indenter particles are in that grid: their mass is there
    assert G[:, 0].sum() == pytest.approx(Mo.sum(), rel=1e-6)
    assert Mo.sum() > o.N * o.m + 0.9 * len(pts) * 4e-8


def test_positions_after_a_press_match_oracle_and_the_gel_is_pushed():
    T, g, o, pts = pair()
    z0 = g.get_state()["u"][2].cpu().numpy().copy()
    g.step(200, 1e-5)
    assert o.run(200, 1e-5) == 0
    u = g.get_state()
    assert u["status"] == 0
    ug = u["u"].cpu().numpy()
    uo = o.state()[0]
    assert np.abs(ug - uo).max() <= 1e-3
    # the particles under the indenter moved down by a good part of its travel
    top = (u["flags"].cpu().numpy() & 2) > 0
    xy = (uo[:2].T * B.dx + np.array(o.origin[:2]))
    under = top & (np.hypot(xy[:, 0] - POSE[0], xy[:, 1] - POSE[1]) < 0.5e-3)
    assert under.sum() > 4
    drop = (z0[under] - ug[2, under]).mean() * B.dx
    assert drop > 0.2 * 0.25 * 200 * 1e-5


def test_switching_back_to_the_grid_boundary():
    T, g, o, pts = pair()
    g.set_indenter_particles(np.zeros((0, 3), np.float32), 1.0)
    o.set_indenter_particles(np.zeros((0, 3)), 1.0)
    g.step(20, 1e-5)
    assert o.run(20, 1e-5) == 0
    assert np.abs(g.get_state()["u"].cpu().numpy() - o.state()[0]).max() <= 1e-3


def test_point_cloud_density_against_the_grid_boundary():
    """The same 0.5 mm sphere press (R 3 mm, 12 x 12 x 3 mm gel at dx 0.5 mm)
    with the grid-boundary indenter and with heavy indenter particles (Eq. 10)
    sampled at two densities, as in the paper's point-cloud study (Sec. IV-B:
    sparse clouds leave surface defects).  A dense cloud (16 points per cell
    volume) carries the surface down to most of the press depth, deeper than
    the grid boundary (whose node-by-node decision holds the surface back by
    a fraction of a cell and leaves a stepped contact, rough at the node
    spacing); a sparse cloud (0.2 per cell volume, 13 points) lets the gel
    slip between its points and stops far short."""
    import paper_2301_08343_gb300 as T
    b = W.Block(24, 24, 6, 0.5e-3, seed=3)
    Rs, depth, n, dt = 3e-3, 0.5e-3, 500, 1e-5
    z_top = b.nz * b.dx
    pose = (b.nx * b.dx / 2, b.ny * b.dx / 2, z_top + Rs, 1, 0, 0, 0)
    vel = (0, 0, -depth / (n * dt), 0, 0, 0)
    win = W.top_window(b)
    cap = math.pi * 1.0e-3 ** 2 * (3 * Rs - 1.0e-3) / 3  # the sampled 1 mm cap

    def press(per_cell=None):
        g = T.Tacchi(b.extent_m, b.dx, b.E, b.nu, b.rho, seed=b.seed)
        g.set_indenter(T.IndenterKind.SPHERE, (Rs,), pose, vel)
        if per_cell:
            pts = W.indenter_points("sphere", (Rs,), max(8, int(per_cell * cap / b.dx ** 3)), seed=1,
                                    reach=1.0e-3).astype(np.float32)
            g.set_indenter_particles(pts, 1e-5)  # about 640 gel particles' mass each
        g.step(n, dt)
        assert g.status() == 0
        return g.heightmap(64, 64, win).cpu().numpy().astype(np.float64)

    xs = (np.arange(64) + 0.5) * (win[2] - win[0]) / 64
    X, Y = np.meshgrid(xs, xs)
    inside = np.hypot(X - pose[0], Y - pose[1]) < 0.8 * math.sqrt(2 * Rs * depth)

    def rough(H):  # RMS of the 5-point Laplacian over the contact
        L = 4 * H[1:-1, 1:-1] - H[:-2, 1:-1] - H[2:, 1:-1] - H[1:-1, :-2] - H[1:-1, 2:]
        return float(np.sqrt((L[inside[1:-1, 1:-1]] ** 2).mean()))

    Hg, Hd, Hs = press(), press(16.0), press(0.2)
    dg, dd, ds = (z_top - Hg).max(), (z_top - Hd).max(), (z_top - Hs).max()
    assert dd >= 0.85 * depth, dd
    assert dg <= dd - 60e-6, (dg, dd)
    assert ds <= 0.75 * dd, (ds, dd)
    assert rough(Hd) <= 0.6 * rough(Hg), (rough(Hd), rough(Hg))
