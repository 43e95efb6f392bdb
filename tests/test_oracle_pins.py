"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: textbook
definitions evaluated differently, closed forms, conservation laws, special
cases with hand-derived answers and published generator output.  They run on
the CPU (no GPU marker).
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def textbook_bspline(d):
    """Quadratic B-spline N(d) of node distance d (cells), piecewise form."""
    a = abs(d)
    if a < 0.5:
        return 0.75 - a * a
    if a < 1.5:
        return 0.5 * (1.5 - a) ** 2
    return 0.0


# ---------------------------------------------------------------- weights --
def test_weights_match_textbook_kernel_on_all_nearby_nodes():
    """Sec. III-A: the 27 stencil weights equal N(xi - X_i) for every node,
    and every node outside the stencil has zero weight."""
    rng = np.random.default_rng(1)
    pts = list(rng.uniform(3.0, 9.0, (200, 3)))
    # fractions on the stencil switch points f = 1/2 and f = 3/2 - eps
    pts += [np.array([5.5, 6.0, 7.0]), np.array([5.0, 5.49999999, 5.5000001])]
    for xi in pts:
        base, w = oracle.weights(xi)
        lo = np.floor(xi).astype(int) - 3
        for k in range(lo[2], lo[2] + 7):
            for j in range(lo[1], lo[1] + 7):
                for i in range(lo[0], lo[0] + 7):
                    ref = (textbook_bspline(xi[0] - i) * textbook_bspline(xi[1] - j)
                           * textbook_bspline(xi[2] - k))
                    o = np.array([i, j, k]) - base
                    got = w[o[2], o[1], o[0]] if np.all((o >= 0) & (o < 3)) else 0.0
                    assert abs(got - ref) <= 1e-15, (xi, i, j, k, got, ref)


def test_weights_partition_of_unity_linear_reproduction_and_inertia():
    """sum w = 1, sum w (X_i - x) = 0 and sum w (X_i - x)(X_i - x)^T = I/4
    (cells^2): the last identity is what makes 4/dX^2 the inverse inertia
    in Eqs. 5 and 8."""
    rng = np.random.default_rng(2)
    for xi in rng.uniform(2.0, 20.0, (500, 3)):
        base, w = oracle.weights(xi)
        s, lin, D = 0.0, np.zeros(3), np.zeros((3, 3))
        for k in range(3):
            for j in range(3):
                for i in range(3):
                    d = base + np.array([i, j, k]) - xi
                    s += w[k, j, i]
                    lin += w[k, j, i] * d
                    D += w[k, j, i] * np.outer(d, d)
        assert abs(s - 1.0) < 1e-12
        assert np.abs(lin).max() < 1e-12
        assert np.abs(D - 0.25 * np.eye(3)).max() < 1e-12


# ------------------------------------------------------------ polar/stress --
def test_polar_recovers_rotation_of_random_rotation_times_spd():
    Rs = W.random_rotations(50, 3)
    rng = np.random.default_rng(4)
    for R0 in Rs:
        A = rng.normal(size=(3, 3))
        S0 = A @ A.T + 0.5 * np.eye(3)
        F = R0 @ S0
        R = oracle.polar(F)
        assert np.abs(R - R0).max() < 1e-11
        assert np.abs(R.T @ R - np.eye(3)).max() < 1e-13
        assert abs(np.linalg.det(R) - 1.0) < 1e-13


def test_polar_near_identity_is_accurate():
    """F = I + small rotation generator + small strain: R - I keeps relative
    accuracy (needed for stress at small strain)."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        th = 1e-4
        K = np.array([[0, -1, 0.3], [1, 0, -0.2], [-0.3, 0.2, 0]]) * th
        R0 = np.eye(3) + K + K @ K / 2 + K @ K @ K / 6  # exp(K) to O(th^4)
        U, _, Vt = np.linalg.svd(R0)
        R0 = U @ Vt
        E = rng.normal(size=(3, 3)) * 1e-5
        S0 = np.eye(3) + (E + E.T) / 2
        R = oracle.polar(R0 @ S0)
        assert np.abs(R - R0).max() < 1e-14


def test_stress_closed_forms():
    E, nu = 3.0e5, 0.45
    mu, la = E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))
    # rigid rotation is stress free
    for R0 in W.random_rotations(20, 6):
        assert np.abs(oracle.stress(R0, mu, la)).max() < 1e-9 * mu
    # uniaxial stretch F = diag(s,1,1): R = I, J = s
    for s in (0.7, 0.95, 1.0, 1.1, 1.6):
        tau = oracle.stress(np.diag([s, 1.0, 1.0]), mu, la)
        p = la * s * (s - 1)
        ref = np.diag([2 * mu * (s - 1) * s + p, p, p])
        assert np.abs(tau - ref).max() < 1e-9 * mu
    # equivariance tau(Q F) = Q tau(F) Q^T
    rng = np.random.default_rng(7)
    for Q in W.random_rotations(20, 8):
        F = np.eye(3) + rng.normal(size=(3, 3)) * 0.1
        assert np.abs(oracle.stress(Q @ F, mu, la) - Q @ oracle.stress(F, mu, la) @ Q.T).max() < 1e-8 * mu
    # small strain limit: linear elasticity 2 mu eps + la tr(eps) I
    G = rng.normal(size=(3, 3))
    G = (G + G.T) / 2
    eps = 1e-6
    tau = oracle.stress(np.eye(3) + eps * G, mu, la)
    lin = 2 * mu * eps * G + la * eps * np.trace(G) * np.eye(3)
    assert np.abs(tau - lin).max() < 1e-4 * np.abs(lin).max()


# --------------------------------------------------------------------- P2G --
def small_sim(nx=3, ny=3, nz=2, dx=1e-3, fix_base=False, pad=4, **kw):
    s = oracle.Sim(nx, ny, nz, dx, 3.0e5, 0.45, 1000.0, pad_side=pad, pad_bottom=pad,
                   pad_top=pad, fix_base=fix_base, **kw)
    u0, fl = oracle.lattice(nx, ny, nz, pad, pad, seed=11)
    return s, u0, fl


def test_p2g_matches_node_centric_brute_force():
    """Eqs. 2-5 gathered node by node with the textbook kernel over all
    particles equal the oracle's stencil scatter."""
    s, u0, fl = small_sim(2, 2, 1)
    u, v, Cm, Fm = W.perturbed_state(u0, 12)
    s.set_state(u, v, Cm, Fm, fl)
    dt = 1e-5
    M, MG = s.p2g(dt)
    xi, vv, CC, FF = s.state()
    X = s.node_positions()
    Xc = (X - s.origin[:, None]) / s.dx
    Mb = np.zeros(s.nodes)
    MGb = np.zeros((3, s.nodes))
    for q in range(s.N):
        tau = oracle.stress(FF[:, q].reshape(3, 3), s.mu, s.la)
        Cq = CC[:, q].reshape(3, 3)
        for n in range(s.nodes):
            d = Xc[:, n] - xi[:, q]
            if np.any(np.abs(d) >= 1.5):
                continue
            w = textbook_bspline(d[0]) * textbook_bspline(d[1]) * textbook_bspline(d[2])
            dm = d * s.dx
            Mb[n] += w * s.m
            MGb[:, n] += w * (s.m * vv[:, q] + s.m * Cq @ dm) - dt * 4 / s.dx ** 2 * w * s.V0 * tau @ dm
    assert np.abs(M - Mb).max() <= 1e-13 * np.abs(Mb).max()
    assert np.abs(MG - MGb).max() <= 1e-12 * np.abs(MGb).max()


def test_p2g_mass_momentum_and_angular_momentum_identities():
    """Sum M_i = sum m_p; sum MG_i = sum m_p v_p (the affine and elastic terms
    vanish by linear reproduction); sum X_i x MG_i = sum_p [x_p x m_p v_p +
    m_p dX^2/4 axial(C_p)] since the symmetric stress exerts no torque."""
    s, u0, fl = small_sim(3, 3, 2)
    u, v, Cm, Fm = W.perturbed_state(u0, 13)
    s.set_state(u, v, Cm, Fm, fl)
    M, MG = s.p2g(1e-5)
    xi, vv, CC, _ = s.state()
    x = s.origin[:, None] + xi * s.dx
    assert abs(M.sum() - s.N * s.m) <= 1e-12 * s.N * s.m
    P = s.m * vv.sum(axis=1)
    assert np.abs(MG.sum(axis=1) - P).max() <= 1e-12 * np.abs(s.m * vv).sum()
    X = s.node_positions()
    Lg = np.cross(X.T, MG.T).sum(axis=0)
    C3 = CC.T.reshape(-1, 3, 3)
    ax = np.stack([C3[:, 2, 1] - C3[:, 1, 2], C3[:, 0, 2] - C3[:, 2, 0], C3[:, 1, 0] - C3[:, 0, 1]], 1)
    Lp = (np.cross(x.T, s.m * vv.T) + s.m * s.dx ** 2 / 4 * ax).sum(axis=0)
    scale = np.abs(np.cross(x.T, s.m * vv.T)).sum()
    assert np.abs(Lg - Lp).max() <= 1e-12 * scale


def _rigid_spin_state(s, u0, v0, omega):
    xi = u0.astype(np.float64)
    x = s.origin[:, None] + xi * s.dx
    c = x.mean(axis=1, keepdims=True)
    v = np.array(v0)[:, None] + np.cross(np.array(omega)[None, :], (x - c).T).T
    W_ = np.array([[0, -omega[2], omega[1]], [omega[2], 0, -omega[0]], [-omega[1], omega[0], 0]])
    Cm = np.repeat(W_.reshape(9, 1), s.N, axis=1)
    return v.astype(np.float32), Cm.astype(np.float32)


def test_free_flight_conserves_linear_and_angular_momentum():
    """No boundary active, no gravity: the grid momentum and angular momentum
    after each P2G stay constant over 300 substeps (APIC transfers and a
    symmetric stress conserve both)."""
    s, u0, fl = small_sim(4, 4, 2, pad=8)
    v, Cm = _rigid_spin_state(s, u0, (0.01, -0.02, 0.015), (3.0, -2.0, 5.0))
    s.set_state(u0, v, Cm, None, fl)
    X = s.node_positions()
    dt = 2e-5
    hist = []
    for it in range(300):
        assert s.substep(dt) == 0
        if it in (0, 299):
            M, MG = s.last_grid()
            hist.append((MG.sum(axis=1), np.cross(X.T, MG.T).sum(axis=0)))
    (P0, L0), (P1, L1) = hist
    assert np.abs(P1 - P0).max() <= 1e-12 * np.abs(P0).max()
    assert np.abs(L1 - L0).max() <= 1e-12 * np.abs(L0).max()


def test_uniform_translation_is_exact_and_stress_free():
    s, u0, fl = small_sim(3, 3, 2, pad=6)
    v0 = np.array([0.05, -0.03, 0.02])
    v = np.repeat(v0[:, None], s.N, axis=1).astype(np.float32)
    s.set_state(u0, v, None, None, fl)
    n, dt = 50, 1e-5
    assert s.run(n, dt) == 0
    xi, vv, CC, FF = s.state()
    exp = u0.astype(np.float64) + n * dt * v.astype(np.float64) / s.dx
    assert np.abs(xi - exp).max() < 1e-11
    assert np.abs(vv - v.astype(np.float64)).max() < 1e-12 * np.abs(v0).max()
    assert np.abs(CC).max() < 1e-9
    assert np.abs(FF - np.eye(3).reshape(9, 1)).max() < 1e-13


def test_rotated_configuration_is_stress_free():
    s, u0, fl = small_sim(3, 3, 2)
    R0 = W.random_rotations(1, 9)[0]
    Fm = np.repeat((R0 - np.eye(3)).reshape(9, 1), s.N, axis=1).astype(np.float32)
    s.set_state(u0, None, None, Fm, fl)
    M, MG = s.p2g(1e-5)
    # the stress of a strain of 1e-3 for comparison
    Fs = np.repeat((np.eye(3) * 1e-3).reshape(9, 1), s.N, axis=1).astype(np.float32)
    s.set_state(u0, None, None, Fs, fl)
    _, MGs = s.p2g(1e-5)
    assert np.abs(MG).max() <= 1e-5 * np.abs(MGs).max()  # FP32 rounding of R0 only


# ------------------------------------------------------------------- G2P --
def _affine_field(s, v0, G, Xref):
    """Grid velocity V(X) = v0 + G (X - Xref) on every node, [3][nodes]."""
    X = s.node_positions()
    return v0[:, None] + G @ (X - Xref[:, None])


def _affine_case(fix_base):
    s, u0, fl = small_sim(4, 4, 3, dx=1e-3, fix_base=fix_base, pad=5)
    rng = np.random.default_rng(21)
    G = rng.uniform(-150.0, 150.0, (3, 3))        # 1/s, not symmetric
    v0 = np.array([0.03, -0.02, 0.015])            # m/s
    Xref = s.origin + 0.5 * np.array(s.G) * s.dx
    Fm = (0.15 * rng.standard_normal((9, s.N))).astype(np.float32)  # F0 - I, order matters
    s.set_state(u0, None, None, Fm, fl)
    x0 = s.origin[:, None] + u0.astype(np.float64) * s.dx
    F0 = Fm.T.astype(np.float64).reshape(-1, 3, 3) + np.eye(3)
    return s, u0, fl, G, v0, Xref, x0, F0


def test_g2p_reproduces_an_affine_grid_velocity_exactly():
    """Eqs. 7-8 with quadratic B-splines reproduce an affine field exactly:
    v_p = V(x_p) (partition of unity and linear reproduction) and
    C_p = (4/dX^2) sum_i w V_i (X_i - x_p)^T = G, because sum_i w (X_i - x_p)
    (X_i - x_p)^T = dX^2 / 4 I.  Eq. 9 then gives F = (I + dt G) F0, in
    that order (G is not symmetric and F0 is a random matrix, so
    F0 (I + dt G) or F0 + dt G differ by far more than the tolerance), and
    Eq. 11 moves x by dt v."""
    s, u0, fl, G, v0, Xref, x0, F0 = _affine_case(False)
    dt = 1e-5
    assert s.g2p(_affine_field(s, v0, G, Xref), dt) == 0
    xi, v, Cm, F = s.state()
    v_exp = v0[:, None] + G @ (x0 - Xref[:, None])
    assert np.abs(v - v_exp).max() <= 1e-13 * np.abs(v_exp).max()
    Cp = Cm.T.reshape(-1, 3, 3)
    assert np.abs(Cp - G[None]).max() <= 1e-11 * np.abs(G).max()
    Fp = F.T.reshape(-1, 3, 3)
    F_exp = np.einsum("ab,pbc->pac", np.eye(3) + dt * G, F0)
    err = np.abs(Fp - F_exp).max()
    assert err <= 1e-13
    wrong_order = np.einsum("pab,bc->pac", F0, np.eye(3) + dt * G)
    assert np.abs(wrong_order - F_exp).max() > 1e6 * max(err, 1e-16)
    assert np.abs((F0 + dt * G[None]) - F_exp).max() > 1e6 * max(err, 1e-16)
    x1 = s.origin[:, None] + xi * s.dx
    assert np.abs(x1 - (x0 + dt * v_exp)).max() <= 1e-15


def test_g2p_base_particles_stop_but_still_deform():
    """Eq. 10: particles of the base set B (flag bit 0) take v = 0 and stay
    put, while C and F follow Eqs. 8-9 like every other particle; particles
    outside B move with the field."""
    s, u0, fl, G, v0, Xref, x0, F0 = _affine_case(True)
    dt = 1e-5
    assert s.g2p(_affine_field(s, v0, G, Xref), dt) == 0
    xi, v, Cm, F = s.state()
    base = (fl & 1) > 0
    assert 0 < base.sum() < s.N
    assert np.all(v[:, base] == 0.0)
    assert np.all(xi[:, base] == u0[:, base].astype(np.float64))
    v_exp = v0[:, None] + G @ (x0 - Xref[:, None])
    assert np.abs(v[:, ~base] - v_exp[:, ~base]).max() <= 1e-13 * np.abs(v_exp).max()
    Cp = Cm.T.reshape(-1, 3, 3)
    assert np.abs(Cp[base] - G[None]).max() <= 1e-11 * np.abs(G).max()
    F_exp = np.einsum("ab,pbc->pac", np.eye(3) + dt * G, F0)
    assert np.abs(F.T.reshape(-1, 3, 3)[base] - F_exp[base]).max() <= 1e-13


def test_box_local_g2p_reproduces_an_affine_grid_velocity_exactly():
    """The box-local substep of oracle/local.py (the judge of the full-size
    sampled parity tests) meets the same affine-field identities."""
    from oracle.local import Local
    s, u0, fl, G, v0, Xref, x0, F0 = _affine_case(True)
    dt = 1e-5
    Vn = _affine_field(s, v0, G, Xref)                   # [3][nodes]
    gx, gy, gz = s.G
    V = Vn.T.reshape(gz, gy, gx, 3)                      # [z][y][x][3]
    L = Local(s.dx, dt, 3.0e5, 0.45, 1000.0)
    fixed = (fl & 1) > 0
    u1, v1, C1, F1 = L.g2p(u0.T.astype(np.float64), F0, fixed, V, np.zeros(3, int))
    v_exp = (v0[:, None] + G @ (x0 - Xref[:, None])).T
    v_exp[fixed] = 0.0
    assert np.abs(v1 - v_exp).max() <= 1e-13 * np.abs(v_exp).max()
    assert np.abs(C1 - G[None]).max() <= 1e-11 * np.abs(G).max()
    F_exp = np.einsum("ab,pbc->pac", np.eye(3) + dt * G, F0)
    assert np.abs(F1 - F_exp).max() <= 1e-13
    assert np.abs(u1 - (u0.T + dt / s.dx * v_exp)).max() <= 1e-12


# -------------------------------------------------------------- grid update --
def test_grid_update_eq6_and_boundaries():
    s, u0, fl = small_sim(4, 4, 3, dx=1e-3, fix_base=True, pad=4)
    u, v, Cm, Fm = W.perturbed_state(u0, 14, disp_cells=0.02)
    s.set_state(u, v, Cm, Fm, fl)
    R = 1.5e-3
    pose = (2e-3, 2e-3, 3e-3 + R - 0.6e-3, 1, 0, 0, 0)
    vel = (0.01, 0.0, -0.2, 0.0, 0.0, 0.0)
    s.set_indenter(oracle.IND_SPHERE, (R,), pose, vel)
    inside = np.array([s.node_inside(i, j, k) for k in range(s.G[2]) for j in range(s.G[1])
                       for i in range(s.G[0])])
    dt = 1e-5
    s.substep(dt)
    M, MG = s.last_grid()
    V = s.last_grid_velocity()
    X = s.node_positions()
    gx, gy, gz = s.G
    k = np.arange(s.nodes) // (gx * gy)
    j = (np.arange(s.nodes) // gx) % gy
    i = np.arange(s.nodes) % gx
    band = (i < 2) | (j < 2) | (k < 2) | (i > gx - 3) | (j > gy - 3) | (k > gz - 3)
    base = k <= 4
    free = ~band & ~base & ~inside
    assert inside.sum() > 0 and (inside & ~base & ~band).sum() > 0
    # Eq. 6 on free nodes with mass, zero on empty free nodes
    has = free & (M > 0)
    assert np.abs(V[:, has] - MG[:, has] / M[has]).max() <= 1e-14 * np.abs(V[:, has]).max()
    assert np.all(V[:, free & (M == 0)] == 0)
    # indenter nodes take the rigid velocity (no angular part here)
    ind = inside & ~base & ~band
    assert np.abs(V[:, ind] - np.array(vel[:3])[:, None]).max() < 1e-15
    assert np.all(V[:, base | band] == 0)
    # the FP32 inside decision agrees with the FP64 geometry off the surface
    d = np.linalg.norm(X - np.array(pose[:3])[:, None], axis=0) / s.dx
    clear = np.abs(d - R / s.dx) > 1e-4
    assert np.array_equal(inside[clear], (d <= R / s.dx)[clear])


def _rot_pose(center, seed):
    R = W.random_rotations(1, seed)[0]
    # quaternion (w, x, y, z) from the rotation matrix
    w = math.sqrt(max(0.0, 1 + R[0, 0] + R[1, 1] + R[2, 2])) / 2
    x = math.copysign(math.sqrt(max(0.0, 1 + R[0, 0] - R[1, 1] - R[2, 2])) / 2, R[2, 1] - R[1, 2])
    y = math.copysign(math.sqrt(max(0.0, 1 - R[0, 0] + R[1, 1] - R[2, 2])) / 2, R[0, 2] - R[2, 0])
    z = math.copysign(math.sqrt(max(0.0, 1 - R[0, 0] - R[1, 1] + R[2, 2])) / 2, R[1, 0] - R[0, 1])
    return tuple(center) + (w, x, y, z), R


@pytest.mark.parametrize("kind", ["sphere", "cylinder", "cone", "prism", "heightmap"])
def test_inside_decision_matches_fp64_geometry(kind):
    s, u0, fl = small_sim(8, 8, 4, dx=0.5e-3, pad=4)
    dx = s.dx
    c = np.array([2e-3, 2e-3, 1.5e-3])
    pose, R = _rot_pose(c, {"sphere": 1, "cylinder": 2, "cone": 3, "prism": 4, "heightmap": 5}[kind])
    X = s.node_positions()
    loc = (R.T @ (X - c[:, None])) / dx  # local coordinates in cells
    hm = None
    if kind == "sphere":
        s.set_indenter(oracle.IND_SPHERE, (1.3e-3,), pose)
        g = np.linalg.norm(loc, axis=0) - 1.3e-3 / dx
        ref = g <= 0
    elif kind == "cylinder":
        s.set_indenter(oracle.IND_CYLINDER, (0.9e-3, 1.7e-3), pose)
        g = np.maximum(np.abs(loc[0]) - 1.7e-3 / dx, np.hypot(loc[1], loc[2]) - 0.9e-3 / dx)
        ref = g <= 0
    elif kind == "cone":
        th, h = math.radians(35), 2.0e-3
        s.set_indenter(oracle.IND_CONE, (th, h), pose)
        g = np.maximum.reduce([-loc[2], loc[2] - h / dx, np.hypot(loc[0], loc[1]) - math.tan(th) * loc[2]])
        ref = g <= 0
    elif kind == "prism":
        th, L, h = math.radians(40), 1.6e-3, 1.8e-3
        s.set_indenter(oracle.IND_PRISM, (th, L, h), pose)
        g = np.maximum.reduce([np.abs(loc[1]) - L / dx, -loc[2], loc[2] - h / dx,
                               np.abs(loc[0]) - math.tan(th) * loc[2]])
        ref = g <= 0
    else:
        n, pix = 16, 0.25e-3
        cc = (np.arange(n) + 0.5 - n / 2) * pix
        a, b = 0.4e-3, 0.1
        hmap = np.repeat((a + b * cc)[None, :], n, axis=0)  # linear in x: exact bilinear
        hm = hmap.astype(np.float32)
        s.set_indenter(oracle.IND_HEIGHTMAP, (1.0e-3,), pose, hm=hm, hm_pixel=pix)
        half = n * pix / 2 / dx
        hloc = (a + b * loc[0] * dx) / dx
        g = np.maximum.reduce([np.abs(loc[0]) - half, np.abs(loc[1]) - half,
                               -hloc - loc[2], loc[2] - 1.0e-3 / dx])
        ref = g <= 0
    got = np.array([s.node_inside(i, j, k) for k in range(s.G[2]) for j in range(s.G[1])
                    for i in range(s.G[0])])
    clear = np.abs(g) > 1e-3
    assert ref.sum() > 10
    assert np.array_equal(got[clear], ref[clear])


def test_indenter_pose_advances_with_velocity():
    s, u0, fl = small_sim(2, 2, 2)
    s.set_state(u0, flags=fl)
    pose = (1e-3, 1e-3, 9e-3, 1, 0, 0, 0)
    w = np.array([0.0, 0.0, 2.0])
    s.set_indenter(oracle.IND_SPHERE, (1e-3,), pose, (0.1, 0, -0.2, *w))
    n, dt = 40, 1e-5
    s.run(n, dt)
    p = s.pose()
    assert np.allclose(p[:3], np.array(pose[:3]) + n * dt * np.array([0.1, 0, -0.2]), atol=1e-15)
    ang = 2.0 * n * dt
    assert np.allclose(p[3:], [math.cos(ang / 2), 0, 0, math.sin(ang / 2)], atol=1e-14)


# ----------------------------------------------------------------- lattice --
def test_splitmix64_matches_published_sequence():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    for k, val in rows:
        assert oracle.splitmix64_at(0, int(k)) == int(val, 16)


def test_lattice_is_stratified_and_flags_count():
    nx, ny, nz, pad, padb = 5, 4, 3, 4, 3
    u, fl = oracle.lattice(nx, ny, nz, pad, padb, seed=3)
    N = 8 * nx * ny * nz
    assert u.shape == (3, N)
    p = np.arange(N)
    s = p % 8
    cell = p // 8
    cx, cy, cz = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    sub = np.stack([s & 1, (s >> 1) & 1, s >> 2])
    lo = np.stack([cx + pad, cy + pad, cz + padb]) + sub * 0.5
    assert np.all(u >= lo) and np.all(u <= lo + 0.5)
    assert (fl & 1).sum() == 8 * nx * ny and np.all((fl & 1) == (cz == 0))
    assert ((fl & 2) > 0).sum() == 4 * nx * ny
    frac = (u - lo) * 2.0
    assert abs(frac.mean() - 0.5) < 0.03 and frac.min() >= 0 and frac.max() < 1
    u2, _ = oracle.lattice(nx, ny, nz, pad, padb, seed=3, jitter=False)
    assert np.array_equal(u2, (lo + 0.25).astype(np.float32))


# --------------------------------------------------------------- height map --
def hm_setup(nx=8, ny=8, dx=1e-3):
    s, u0, fl = small_sim(nx, ny, 2, dx=dx, pad=4)
    s.set_rest(u0)
    return s, u0, fl


def test_heightmap_rest_and_uniform_shift():
    s, u0, fl = hm_setup()
    win = (0.0, 0.0, 8e-3, 8e-3)
    s.set_state(u0, flags=fl)
    H = s.heightmap(win, 32, 32)
    assert np.all(H == s.z_top)
    u = u0.copy()
    u[2] += np.float32(0.25)
    s.set_state(u, flags=fl)
    H = s.heightmap(win, 32, 32)
    assert np.abs(H - (s.z_top + 0.25 * s.dx)).max() < 1e-15


def test_heightmap_single_raised_particle_covers_its_disc():
    s, u0, fl = hm_setup()
    win = (0.0, 0.0, 8e-3, 8e-3)
    surf = np.nonzero(fl & 2)[0]
    xy = u0[:2, surf].astype(np.float64)
    q = surf[np.argmin(np.abs(xy[0] - 8.0) + np.abs(xy[1] - 8.3))]  # an interior one
    u = u0.copy()
    u[2, q] = u0[2, q] + np.float32(0.3)
    s.set_state(u, flags=fl)
    w = h = 64
    H = s.heightmap(win, w, h)
    pxc = 8e-3 / w / s.dx
    cc = (np.arange(w) + 0.5) * pxc + 4  # pixel centres in cells (origin at -4 cells)
    QX, QY = np.meshgrid(cc, cc, indexing="xy")
    d2 = (QX - u0[0, q]) ** 2 + (QY - u0[1, q]) ** 2
    val = s.z_top + s.dx * (np.float64(u[2, q]) - np.float64(u0[2, q]))
    clear = np.abs(d2 - 0.25) > 1e-4
    assert np.array_equal((H > s.z_top)[clear], (d2 <= 0.25)[clear])
    assert np.abs(H[d2 <= 0.2] - val).max() < 1e-15


def test_heightmap_hole_fill_reaches_fill_radius_only():
    s, u0, fl = hm_setup()
    u = u0.copy()
    u[2] += np.float32(0.25)
    s.set_state(u, flags=fl)
    # window 3 cells wider than the block on every side; 4 pixels per cell
    win = (-3e-3, -3e-3, 11e-3, 11e-3)
    w = h = 56
    R = 3
    H = s.heightmap(win, w, h, fill_radius=R)
    surf = np.nonzero(fl & 2)[0]
    cc = (np.arange(w) + 0.5) * 0.25 + 1.0  # cells (window x0 = -3 mm = cell 1)
    QX, QY = np.meshgrid(cc, cc, indexing="xy")
    cov = np.zeros((h, w), bool)
    for q in surf:
        cov |= (QX - u0[0, q]) ** 2 + (QY - u0[1, q]) ** 2 <= 0.25
    near = np.zeros_like(cov)
    for dr in range(-R, R + 1):
        for dc in range(-R, R + 1):
            sh = np.zeros_like(cov)
            r0, r1 = max(0, dr), h + min(0, dr)
            c0, c1 = max(0, dc), w + min(0, dc)
            sh[r0:r1, c0:c1] = cov[r0 - dr:r1 - dr, c0 - dc:c1 - dc]
            near |= sh
    shifted = s.z_top + 0.25 * s.dx
    assert np.abs(H[near] - shifted).max() < 1e-15
    assert np.all(H[~near] == s.z_top)
    assert (~near).sum() > 0 and (near & ~cov).sum() > 0


# ----------------------------------------------------------------- shading --
def lights():
    return W.default_lights()


def _rp(**over):
    d = dict(lights())
    d.update(over)
    return oracle.render_params(d["n_lights"], d["dirs"], d["diffuse"], d["specular"],
                                d["ambient"], d["ka"], d["kd"], d["ks"], d["alpha"])


def test_shading_flat_surface_is_the_eq12_scalar():
    """Flat H: N = V = (0,0,-1), so L.N = R.V = -L_z for every light."""
    L = lights()
    rp = _rp()
    H = np.full((20, 30), 3e-3)
    img = oracle.shade(H, 1e-4, 1e-4, 3e-3, rp)
    exp = np.array(L["ambient"]) * L["ka"]
    for m in range(3):
        c = -L["dirs"][m][2]
        exp = exp + L["kd"] * c * np.array(L["diffuse"][m]) + L["ks"] * c ** L["alpha"] * np.array(L["specular"][m])
    exp = np.clip(exp, 0, 1)
    assert np.abs(img - exp).max() < 1e-15


def test_shading_normal_from_central_differences_is_exact_for_quadratics():
    """Eq. 14: a paraboloid dimple D = d0 - r^2/(2 Rc) has central-difference
    gradients equal to its analytic gradient, so interior pixels see
    N = normalize(-x/Rc, -y/Rc, -1)."""
    w, h, pix, Rc, z_top = 40, 30, 1e-4, 5e-3, 3e-3
    x = (np.arange(w) - w / 2) * pix
    y = (np.arange(h) - h / 2) * pix
    XX, YY = np.meshgrid(x, y, indexing="xy")
    D = 0.5e-3 - (XX ** 2 + YY ** 2) / (2 * Rc)
    H = z_top - D
    L = lights()
    rp = _rp()
    img = oracle.shade(H, pix, pix, z_top, rp)
    N = np.stack([-XX / Rc, -YY / Rc, -np.ones_like(XX)], -1)
    N /= np.linalg.norm(N, axis=-1, keepdims=True)
    exp = np.zeros((h, w, 3)) + np.array(L["ambient"]) * L["ka"]
    V = np.array([0, 0, -1.0])
    for m in range(3):
        Ld = np.array(L["dirs"][m])
        LN = N @ Ld
        Rv = 2 * LN[..., None] * N - Ld
        RV = Rv @ V
        exp += L["kd"] * np.maximum(LN, 0)[..., None] * np.array(L["diffuse"][m])
        exp += L["ks"] * (np.maximum(RV, 0) ** L["alpha"])[..., None] * np.array(L["specular"][m])
    exp = np.clip(exp, 0, 1)
    assert np.abs(img[1:-1, 1:-1] - exp[1:-1, 1:-1]).max() < 1e-12


def test_shading_slope_toward_light_brightens_that_channel():
    """A light from +x (red) lights a surface whose depth grows with x more
    than a flat one; a light from -x would darken (sign convention of N)."""
    d = lights()
    d["dirs"] = [(math.cos(0.5), 0.0, -math.sin(0.5))]
    d["diffuse"] = [(1.0, 0.0, 0.0)]
    d["specular"] = [(0.0, 0.0, 0.0)]
    d["n_lights"] = 1
    rp = oracle.render_params(1, d["dirs"], d["diffuse"], d["specular"], d["ambient"],
                              0.0, 1.0, 0.0, 5.0)
    w = h = 16
    pix = 1e-4
    XX = np.meshgrid(np.arange(w) * pix, np.arange(h) * pix, indexing="xy")[0]
    flat = oracle.shade(np.full((h, w), 3e-3), pix, pix, 3e-3, rp)[5, 5, 0]
    up = oracle.shade(3e-3 - 0.2 * XX, pix, pix, 3e-3, rp)[5, 5, 0]
    down = oracle.shade(3e-3 + 0.2 * XX, pix, pix, 3e-3, rp)[5, 5, 0]
    assert up > flat > down


# ---------------------------------------------------------------------------
# Indenter represented by particles (Eq. 10, p in I)

def _particle_indenter_sim(w):
    s = oracle.Sim(6, 6, 2, 0.5e-3, 3.0e5, 0.45, 1000.0)
    u, fl = oracle.lattice(6, 6, 2, 4, 3, 5, True)
    s.set_state(u)
    pts = W.indenter_points("sphere", (1.2e-3,), 400, seed=3, reach=0.6e-3)
    pose = (1.5e-3, 1.4e-3, 1.0e-3 + 1.2e-3 - 0.2e-3, math.cos(0.2), 0.0, math.sin(0.2) * 0.6, math.sin(0.2) * 0.8)
    vel = (0.05, -0.02, -0.3) + tuple(w)
    s.set_indenter(oracle.IND_SPHERE, (1.2e-3,), pose, vel)
    return s, pts, pose, vel


def test_particle_indenter_adds_its_mass_momentum_and_angular_momentum():
    # Indenter particles add m_I per particle (partition of unity), m_I v_p
    # in total (sum_i w (X_i - x) = 0) and, about the indenter centre c,
    # m_I (r_p x v_p + dX^2 / 2 w) each: sum_i w d x (w x d) = (tr D - D) w
    # with D = sum_i w d d^T = dX^2 / 4 I for the quadratic B-spline.
    w = (40.0, -25.0, 60.0)
    s, pts, pose, vel = _particle_indenter_sim(w)
    dt, mI, dx = 1e-5, 2.5e-8, 0.5e-3
    m0, g0 = s.p2g(dt)
    s.set_indenter_particles(pts, mI)
    m1, g1 = s.p2g(dt)
    dm, dg = m1 - m0, g1 - g0
    qw, qx, qy, qz = pose[3:]
    Rm = np.array([[1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)],
                   [2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)],
                   [2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)]])
    r = pts @ Rm.T
    v = np.array(vel[:3]) + np.cross(np.array(w), r)
    assert dm.sum() == pytest.approx(len(pts) * mI, rel=1e-12)
    assert np.allclose(dg.sum(axis=1), mI * v.sum(axis=0), rtol=1e-10, atol=1e-20)
    X = s.node_positions().T
    L = np.cross(X - np.array(pose[:3]), dg.T).sum(axis=0)
    Lp = mI * (np.cross(r, v).sum(axis=0) + len(pts) * dx * dx / 2 * np.array(w))
    assert np.allclose(L, Lp, rtol=1e-9, atol=1e-24)


def test_particle_indenter_leaves_grid_nodes_to_the_momentum():
    # with particles, nodes inside the shape take MG / M like any other node
    s, pts, pose, vel = _particle_indenter_sim((0.0, 0.0, 0.0))
    s.set_indenter_particles(pts, 2.5e-8)
    s.substep(1e-5)
    m, g = s.last_grid()
    V = s.last_grid_velocity()
    G = s.G

    def ijk(n):
        return n % G[0], (n // G[0]) % G[1], n // (G[0] * G[1])

    def interior(n):  # clear of the padding band and of the fixed base
        i, j, k = ijk(n)
        return min(i, j) >= 2 and k > 3 and i <= G[0] - 3 and j <= G[1] - 3 and k <= G[2] - 3

    inside = [n for n in range(s.nodes) if m[n] > 0 and interior(n) and s.node_inside(*ijk(n))]
    assert len(inside) > 5
    for n in inside:
        assert np.allclose(V[:, n], g[:, n] / m[n], rtol=1e-12, atol=0)
    # nodes the elastomer's mass also reaches move slower than the indenter
    assert any(not np.allclose(V[:, n], vel[:3]) for n in inside)
    # back to the grid boundary: the nodes inside take the rigid velocity
    s.set_indenter_particles(np.zeros((0, 3)), 1.0)
    s.substep(1e-5)
    V = s.last_grid_velocity()
    n = [q for q in range(s.nodes) if interior(q) and s.node_inside(*ijk(q))][0]
    assert np.allclose(V[:, n], vel[:3], rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------ slip contact --
def _shape_phi(kind, params, pose, hm=None, hm_pixel=None):
    """The shapes' defining inequalities (inside where phi <= 0 near the
    contact surface), as the C ABI header states them: sphere |X - c| - R;
    cylinder (axis local x) sqrt(y_l^2 + z_l^2) - R; cone sqrt(x_l^2 + y_l^2)
    - tan(a) z_l; prism |x_l| - tan(a) z_l; height map -z_l - h(x_l, y_l)
    with h the bilinear interpolant of the samples (the edge samples extended
    beyond the outermost sample centres)."""
    q = np.asarray(pose[3:], float)
    q = q / np.linalg.norm(q)
    w_, x_, y_, z_ = q
    Rm = np.array([[1 - 2 * (y_ * y_ + z_ * z_), 2 * (x_ * y_ - w_ * z_), 2 * (x_ * z_ + w_ * y_)],
                   [2 * (x_ * y_ + w_ * z_), 1 - 2 * (x_ * x_ + z_ * z_), 2 * (y_ * z_ - w_ * x_)],
                   [2 * (x_ * z_ - w_ * y_), 2 * (y_ * z_ + w_ * x_), 1 - 2 * (x_ * x_ + y_ * y_)]])
    c = np.asarray(pose[:3], float)

    def phi(X):
        l = Rm.T @ (X - c)
        if kind == oracle.IND_SPHERE:
            return np.linalg.norm(X - c) - params[0]
        if kind == oracle.IND_CYLINDER:
            return math.hypot(l[1], l[2]) - params[0]
        if kind == oracle.IND_CONE:
            return math.hypot(l[0], l[1]) - math.tan(params[0]) * l[2]
        if kind == oracle.IND_PRISM:
            return abs(l[0]) - math.tan(params[0]) * l[2]
        h_, w = hm.shape
        fx, fy = l[0] / hm_pixel + (w / 2 - 0.5), l[1] / hm_pixel + (h_ / 2 - 0.5)
        fx, fy = min(max(fx, 0.0), w - 1.0), min(max(fy, 0.0), h_ - 1.0)  # edge samples extend outward
        ix, iy = min(int(math.floor(fx)), w - 2), min(int(math.floor(fy)), h_ - 2)
        tx, ty = fx - ix, fy - iy
        hv = ((hm[iy, ix] * (1 - tx) + hm[iy, ix + 1] * tx) * (1 - ty)
              + (hm[iy + 1, ix] * (1 - tx) + hm[iy + 1, ix + 1] * tx) * ty)
        return -l[2] - hv
    return phi


@pytest.mark.parametrize("kind", ["sphere", "cylinder", "cone", "prism", "heightmap"])
def test_slip_contact_removes_only_the_velocity_into_the_indenter(kind):
    """Slip contact (reading c8): a node inside the indenter that holds mass
    keeps its velocity V except the part that moves into the indenter,
    relative to it: V <- W + q - min(0, q.n) n with q = V - W, W the rigid
    velocity and n the unit outward normal, here the gradient of the shape's
    defining function by central differences.  A uniform flow v0 with F = I
    and C = 0 puts MG = M v0 on every node, so V = v0 before the condition;
    sticky contact sets W instead."""
    nx = ny = 8
    nz, dx = 4, 0.5e-3
    u0, fl = oracle.lattice(nx, ny, nz, 4, 3, seed=3)
    rng = np.random.default_rng(4)
    v0 = np.array([0.03, -0.02, 0.05])
    v = np.repeat(v0[:, None], u0.shape[1], axis=1).astype(np.float32)
    z_top = nz * dx
    c = (nx * dx / 2 + 0.13e-3, ny * dx / 2 - 0.07e-3)
    hm, hm_pixel = None, 0.0
    if kind == "sphere":
        k, params, tip = oracle.IND_SPHERE, (1.3e-3,), 1.3e-3
        quat = (1.0, 0.0, 0.0, 0.0)
    elif kind == "cylinder":
        k, params, tip = oracle.IND_CYLINDER, (0.9e-3, 1.5e-3), 0.9e-3
        quat = (math.cos(0.2), 0.0, 0.0, math.sin(0.2))     # yaw: the axis stays horizontal
    elif kind == "cone":
        k, params, tip = oracle.IND_CONE, (math.radians(40), 1.5e-3), 0.0
        quat = (math.cos(0.05), math.sin(0.05), 0.0, 0.0)
    elif kind == "prism":
        k, params, tip = oracle.IND_PRISM, (math.radians(50), 1.5e-3, 1.5e-3), 0.0
        quat = (math.cos(0.3), 0.0, 0.0, math.sin(0.3))
    else:
        k, tip = oracle.IND_HEIGHTMAP, 0.6e-3
        hm_pixel = 0.2e-3
        yy, xx = np.mgrid[0:16, 0:16]
        hm = (0.6e-3 * np.exp(-((xx - 7.3) ** 2 + (yy - 8.1) ** 2) / 18.0)).astype(np.float32)
        params = (0.5e-3,)
        quat = (math.cos(0.15), 0.0, 0.0, math.sin(0.15))
    pose = (c[0], c[1], z_top + tip - 0.7e-3) + quat
    vel = (0.01, -0.02, -0.1, 0.0, 0.0, 3.0)
    runs = {}
    for slip in (False, True):
        s = oracle.Sim(nx, ny, nz, dx, 3e5, 0.45, 1000.0, fix_base=True, slip=slip)
        s.set_state(u0, v, None, None, fl)
        s.set_indenter(k, params, pose, vel, hm=hm, hm_pixel=hm_pixel)
        assert s.substep(1e-6) == 0
        runs[slip] = (s, s.last_grid_velocity(), s.last_grid()[0])
    s, Vs, M = runs[True]
    _, Vk, _ = runs[False]
    X = s.node_positions()
    # the method keeps the height samples as FP32 heights in grid cells
    hm_used = None if hm is None else (hm.astype(np.float64) / dx).astype(np.float32).astype(np.float64) * dx
    phi = _shape_phi(k, params, pose, hm_used, hm_pixel)
    gx, gy, gz = s.G
    checked = moved_in = 0
    for e in range(s.nodes):
        i, j, kk = e % gx, (e // gx) % gy, e // (gx * gy)
        if not s.node_inside(i, j, kk) or kk <= 3 or M[e] <= 0.0:
            continue
        Xe = X[:, e]
        r = Xe - np.asarray(pose[:3])
        Wv = np.asarray(vel[:3]) + np.cross(np.asarray(vel[3:]), r)
        assert np.allclose(Vk[:, e], Wv, rtol=0, atol=1e-15)          # sticky
        h = 1e-7
        grad = np.array([(phi(Xe + h * ea) - phi(Xe - h * ea)) / (2 * h) for ea in np.eye(3)])
        if np.linalg.norm(grad) < 0.5:
            continue  # on an axis or edge: the normal is undefined there
        n = grad / np.linalg.norm(grad)
        qv = v0 - Wv
        vn = qv @ n
        exp = Wv + qv - min(0.0, vn) * n
        assert np.abs(Vs[:, e] - exp).max() <= 1e-8 * max(1.0, np.abs(exp).max()), (kind, e, Vs[:, e], exp)
        checked += 1
        moved_in += vn < 0
    assert checked >= 5 and 0 < moved_in < checked + 1
