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
