"""The box-local FP64 substeps used by the full-size sampled parity test
agree with the oracle's own whole-grid substeps: two substeps of a block
with a smooth random velocity field, random affine velocities and random
F - I, free base, no indenter; the grid of the second P2G at an interior
node and the state of the particles whose stencils the box covers."""
import numpy as np

import oracle
from oracle.local import Local, velocity


def test_box_local_substeps_equal_the_oracle():
    nx = ny = nz = 18
    dx, dt, E, nu, rho = 1e-3, 2e-6, 3e5, 0.45, 1000.0
    o = oracle.Sim(nx, ny, nz, dx, E, nu, rho, fix_base=False)
    u0, _ = oracle.lattice(nx, ny, nz, 4, 3, seed=5)
    N = u0.shape[1]
    rng = np.random.default_rng(1)
    v = np.vstack([0.5 * np.sin(u0[0] * 0.3), 0.3 * np.cos(u0[2] * 0.25),
                   0.2 * np.sin(u0[0] * 0.15 + u0[1] * 0.1)]).astype(np.float32)
    Cm = (50 * rng.standard_normal((9, N))).astype(np.float32)
    Fm = (0.02 * rng.standard_normal((9, N))).astype(np.float32)
    o.set_state(u0, v, Cm, Fm, np.zeros(N, np.uint8))
    assert o.run(2, dt) == 0
    Mo, MGo = o.last_grid()
    xi, _, _, Fo = o.state()
    G0, G1, _ = o.G
    L = Local(dx, dt, E, nu, rho)
    c = np.array([13, 13, 12])
    lo, hi = c - 6, c + 6
    up = u0.T.astype(np.float64)
    base = np.floor(up - 0.5).astype(int)
    sel = np.all((base >= lo) & (base <= hi), axis=1)
    ids = np.nonzero(sel)[0]
    shape = tuple((hi - lo + 3)[::-1])
    F0 = Fm.T[sel].astype(np.float64).reshape(-1, 3, 3) + np.eye(3)
    M0, MG0 = L.p2g(up[sel], v.T[sel].astype(np.float64), Cm.T[sel].astype(np.float64).reshape(-1, 3, 3),
                    F0, lo, shape)
    inner = np.all((base[sel] >= lo + 2) & (base[sel] <= hi - 2), axis=1)
    fixed = np.zeros(len(ids), bool)
    u1, v1, C1, F1 = L.g2p(up[sel][inner], F0[inner], fixed[inner], velocity(M0, MG0), lo)
    M1, MG1 = L.p2g(u1, v1, C1, F1, lo, shape)
    e = (c[2] * G1 + c[1]) * G0 + c[0]
    i0 = tuple((c - lo)[::-1])
    assert M1[i0] > 0 and abs(M1[i0] - Mo[e]) <= 1e-14 * Mo[e]
    assert np.abs(MG1[i0] - MGo[:, e]).max() <= 1e-12 * np.abs(MGo[:, e]).max()
    b1 = np.floor(u1 - 0.5).astype(int)
    core = np.all((b1 >= lo + 5) & (b1 <= hi - 5), axis=1)
    u2, _, _, F2 = L.g2p(u1[core], F1[core], fixed[inner][core], velocity(M1, MG1), lo)
    got = ids[inner][core]
    assert len(got) >= 100
    assert np.abs(xi.T[got] - u2).max() <= 1e-12
    assert np.abs(Fo.T[got].reshape(-1, 3, 3) - F2).max() <= 1e-12


def test_box_local_substeps_with_boundary_conditions_equal_the_oracle():
    """The same with every grid boundary condition inside the box: a sphere
    pressed into a thin block with a fixed base (its nodes and its base-set
    particles) and the padding band below the base; the box-local grid
    velocity takes the oracle's own inside decision at each substep's pose."""
    from oracle.local import grid_velocity
    nx = ny = 18
    nz, pad = 6, 3
    dx, dt, E, nu, rho = 1e-3, 2e-6, 3e5, 0.45, 1000.0
    R = 4e-3
    o = oracle.Sim(nx, ny, nz, dx, E, nu, rho, pad_side=4, pad_bottom=pad, pad_top=4, fix_base=True)
    u0, fl = oracle.lattice(nx, ny, nz, 4, pad, seed=5)
    N = u0.shape[1]
    rng = np.random.default_rng(2)
    v = (0.05 * rng.standard_normal((3, N))).astype(np.float32)
    Fm = (0.01 * rng.standard_normal((9, N))).astype(np.float32)
    o.set_state(u0, v, None, Fm, fl)
    pose0 = (nx * dx / 2 + 0.3e-3, ny * dx / 2 - 0.2e-3, nz * dx + R - 1.5e-3, 1.0, 0.0, 0.0, 0.0)
    vel = (0.1, 0.0, -0.8, 0.0, 0.0, 40.0)
    o.set_indenter(oracle.IND_SPHERE, (R,), pose0, vel)
    probe = oracle.Sim(nx, ny, nz, dx, E, nu, rho, pad_side=4, pad_bottom=pad, pad_top=4, fix_base=True)
    poses = []
    for _ in range(2):
        poses.append(o.pose())
        assert o.substep(dt) == 0
    Mo, MGo = o.last_grid()
    xi, _, _, Fo = o.state()
    G0, G1, _ = o.G

    def inside_at(pose):
        probe.set_indenter(oracle.IND_SPHERE, (R,), pose, vel)
        return probe.node_inside

    L = Local(dx, dt, E, nu, rho)
    bc = dict(dx=dx, origin=o.origin, vel=vel, base_k=pad)
    up = u0.T.astype(np.float64)
    base = np.floor(up - 0.5).astype(int)
    seen_inside = seen_fixed = False
    for c in (np.array([13, 13, 8]), np.array([13, 13, 4])):   # under the indenter; at the base
        lo, hi = c - 6, c + 6
        sel = np.all((base >= lo) & (base <= hi), axis=1)
        ids = np.nonzero(sel)[0]
        fixed = (fl[sel] & 1) > 0
        shape = tuple((hi - lo + 3)[::-1])
        F0 = Fm.T[sel].astype(np.float64).reshape(-1, 3, 3) + np.eye(3)
        M0, MG0 = L.p2g(up[sel], v.T[sel].astype(np.float64), np.zeros((len(ids), 3, 3)), F0, lo, shape)
        V0 = grid_velocity(M0, MG0, lo, o.G, inside=inside_at(poses[0]), pose=poses[0], **bc)
        inner = np.all((base[sel] >= lo + 2) & (base[sel] <= hi - 2), axis=1)
        u1, v1, C1, F1 = L.g2p(up[sel][inner], F0[inner], fixed[inner], V0, lo)
        M1, MG1 = L.p2g(u1, v1, C1, F1, lo, shape)
        e = (c[2] * G1 + c[1]) * G0 + c[0]
        i0 = tuple((c - lo)[::-1])
        assert M1[i0] > 0 and abs(M1[i0] - Mo[e]) <= 1e-13 * Mo[e]
        assert np.abs(MG1[i0] - MGo[:, e]).max() <= 1e-12 * np.abs(MGo[:, e]).max()
        V1 = grid_velocity(M1, MG1, lo, o.G, inside=inside_at(poses[1]), pose=poses[1], **bc)
        b1 = np.floor(u1 - 0.5).astype(int)
        core = np.all((b1 >= lo + 5) & (b1 <= hi - 5), axis=1)
        u2, _, _, F2 = L.g2p(u1[core], F1[core], fixed[inner][core], V1, lo)
        got = ids[inner][core]
        assert len(got) >= 100
        assert np.abs(xi.T[got] - u2).max() <= 1e-12
        assert np.abs(Fo.T[got].reshape(-1, 3, 3) - F2).max() <= 1e-12
        # nodes of the core's stencils inside the indenter; fixed particles in the core
        seen_inside |= any(inside_at(poses[1])(i, j, k) for i in range(c[0] - 1, c[0] + 4)
                           for j in range(c[1] - 1, c[1] + 4) for k in range(c[2] - 1, c[2] + 4))
        seen_fixed |= bool(fixed[inner][core].any())
    assert seen_inside and seen_fixed
