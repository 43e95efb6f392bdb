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
