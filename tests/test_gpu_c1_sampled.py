"""Parity at the full GelSight-scale workload in the launch configuration the
benchmark times (24,576,000 particles, 8 x 8 x 4 sort blocks, the fused
G2P + P2G transfer), on outputs that the oracle's per-particle routines can
compute one by one.

After 200 substeps of a fast sphere press (0.5 mm at 2.5 m/s) the GPU state
S is read back and two more substeps run on the GPU: the opening P2G of S,
the grid update, the fused transfer (G2P of substep 0, P2G of substep 1),
the grid update and the closing G2P.  Around sampled nodes the same two
substeps are recomputed in FP64 from S over a box of particles large enough
for every value used to be complete: P2G (Eqs. 2-5, the stress from the
oracle's polar decomposition), grid velocity (Eq. 6), G2P, F update and
advection (Eqs. 7-11), P2G again, grid velocity, G2P.  Compared: the grid of
the fused transfer's P2G at the sampled nodes (the c21 reading: max |dMG| /
max |MG| <= 1e-5 over the sample, the same for M), and the particles' state
after the closing G2P: positions to 1e-4 cells (FP32 spacing at 300 cells is
3e-5), F - I to 1e-4 of its largest entry (the FP32 rounding of the 27-term
G2P sums, about 2e-7 per substep).  The nodes are those with the largest
momentum whose whole box is clear of the indenter, the fixed base and the
padding band, plus two boxes where the boundary conditions act: one whose
nodes cut the sphere (rigid indenter velocity on the nodes inside it, decided
by the oracle's FP32 inside test at each substep's pose) and one on the
sensor base (its nodes held at zero and its base-set particles stopped,
Eq. 10).  Also checked at every node: the total grid mass equals N m; and the
640 x 480 frame of the final state against the oracle's height map and
shading."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.local import Local, grid_velocity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def test_c1_two_substeps_at_sampled_nodes_and_particles():
    import paper_2301_08343_gb300 as T
    import oracle
    b, dt = W.C1, W.C1_DT
    dx = b.dx
    g = T.Tacchi(b.extent_m, dx, b.E, b.nu, b.rho, seed=0, pad_side=b.pad_side, pad_bottom=b.pad_bottom,
                 pad_top=b.pad_top)
    assert g.block == (8, 8, 4) and g.threads_per_cell == 1 and g.N == 24_576_000
    R, depth, n = 4e-3, 0.5e-3, 200
    g.set_indenter(T.IndenterKind.SPHERE, (R,), (b.nx * dx / 2, b.ny * dx / 2, g.z_top + R, 1, 0, 0, 0),
                   (0, 0, -depth / (n * dt), 0, 0, 0))
    g.step(n, dt)
    S = g.get_state()
    assert S["status"] == 0
    pose = g.indenter_pose()
    g.step(2, dt)
    S2 = g.get_state()
    assert S2["status"] == 0
    grid = g.get_grid()
    G0, G1, G2 = g.grid
    m = b.rho * dx ** 3 / 8
    # every particle's mass is on the grid
    assert float(grid[:, 0].double().sum()) == pytest.approx(g.N * m, rel=1e-5)

    # nodes with the largest momentum whose box [c - 6, c + 6] is clear of
    # the sphere (by more than a node diagonal), the base and the padding
    org = np.array(g.origin)
    cc = (np.array(pose[:3]) - org) / dx
    MGn = grid[:, 1:].norm(dim=1).reshape(G2, G1, G0)
    kk, jj, ii = torch.meshgrid(torch.arange(G2, device="cuda"), torch.arange(G1, device="cuda"),
                                torch.arange(G0, device="cuda"), indexing="ij")
    dist = torch.sqrt((ii - cc[0]) ** 2 + (jj - cc[1]) ** 2 + (kk - cc[2]) ** 2) - R / dx
    ok = (dist > 6 * math.sqrt(3) + 1) & (kk >= b.pad_bottom + 10) & (ii >= 10) & (jj >= 10) & \
         (ii < G0 - 10) & (jj < G1 - 10) & (kk < G2 - 10)
    score = torch.where(ok, MGn, torch.zeros_like(MGn)).flatten()
    picks = []
    for e in torch.argsort(score, descending=True).tolist():
        c = np.array([e % G0, (e // G0) % G1, e // (G0 * G1)])
        if all(np.abs(c - q).max() > 12 for q in picks):
            picks.append(c)
        if len(picks) == 6:
            break
    assert float(score.max()) > 0
    # the boundary-condition boxes: under the sphere's lowest point, so that
    # nodes of the box lie inside it, and on the base under the press
    k_low = int(math.floor(cc[2] - R / dx))
    c_ind = np.array([int(round(cc[0])) + 3, int(round(cc[1])) - 2, k_low - 1])
    c_base = np.array([int(round(cc[0])) - 5, int(round(cc[1])) + 4, b.pad_bottom + 1])
    picks += [c_ind, c_base]
    vel = (0.0, 0.0, -depth / (n * dt), 0.0, 0.0, 0.0)
    pose1 = tuple(pose[a] + dt * vel[a] if a < 3 else pose[a] for a in range(7))
    assert np.allclose(g.indenter_pose(), [pose1[a] + dt * vel[a] if a < 3 else pose1[a] for a in range(7)],
                       rtol=0, atol=0)
    # the oracle's inside decision depends on dx, the grid origin and the pose only
    probe = oracle.Sim(4, 4, 2, dx, b.E, b.nu, b.rho, b.pad_side, b.pad_bottom, b.pad_top)

    def inside_at(ps):
        probe.set_indenter(oracle.IND_SPHERE, (R,), ps, vel)
        return probe.node_inside

    bc = dict(dx=dx, origin=org, vel=vel, base_k=b.pad_bottom)
    n_inside, n_fixed = 0, 0

    u = S["u"]
    base = torch.floor(u - 0.5).to(torch.int32)
    L = Local(dx, dt, b.E, b.nu, b.rho)
    gM = grid[:, 0].reshape(G2, G1, G0)
    gMG = grid[:, 1:].reshape(G2, G1, G0, 3)
    dM, dMG, sM, sMG, du, dF, sF, nck = 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0
    for c in picks:
        lo, hi = c - 6, c + 6                       # particle base cells of the box
        sel = ((base[0] >= lo[0]) & (base[0] <= hi[0]) & (base[1] >= lo[1]) & (base[1] <= hi[1]) &
               (base[2] >= lo[2]) & (base[2] <= hi[2])).nonzero().flatten()
        ids = sel.cpu().numpy()
        up = u[:, sel].T.double().cpu().numpy()
        vp = S["v"][:, sel].T.double().cpu().numpy()
        Cp = S["C"][:, sel].T.double().cpu().numpy().reshape(-1, 3, 3)
        Fp = S["Fm"][:, sel].T.double().cpu().numpy().reshape(-1, 3, 3) + np.eye(3)
        fixed = (S["flags"][sel].cpu().numpy() & 1) > 0
        shape = tuple((hi - lo + 3)[::-1])
        # substep 0: P2G of S (complete on nodes [lo + 2, hi]), grid velocity
        # with the boundary conditions at the substep's pose
        M0, MG0 = L.p2g(up, vp, Cp, Fp, lo, shape)
        V0 = grid_velocity(M0, MG0, lo, (G0, G1, G2), inside=inside_at(pose), pose=pose, **bc)
        bp = np.floor(up - 0.5).astype(int)
        inner = np.all((bp >= lo + 2) & (bp <= hi - 2), axis=1)  # stencils inside [lo + 2, hi]
        u1, v1, C1, F1 = L.g2p(up[inner], Fp[inner], fixed[inner], V0, lo)
        # substep 1: P2G of S1 (complete on nodes [lo + 5, hi - 3]: no particle
        # moves a cell in a substep)
        M1, MG1 = L.p2g(u1, v1, C1, F1, lo, shape)
        i0 = tuple((c - lo)[::-1])
        gm = float(gM[c[2], c[1], c[0]])
        gmg = gMG[c[2], c[1], c[0]].double().cpu().numpy()
        dM = max(dM, abs(gm - M1[i0]))
        dMG = max(dMG, float(np.abs(gmg - MG1[i0]).max()))
        sM = max(sM, abs(M1[i0]))
        sMG = max(sMG, float(np.abs(MG1[i0]).max()))
        # the closing G2P for the particles whose stencil lies where the
        # substep-1 grid is complete
        V1 = grid_velocity(M1, MG1, lo, (G0, G1, G2), inside=inside_at(pose1), pose=pose1, **bc)
        b1 = np.floor(u1 - 0.5).astype(int)
        core = np.all((b1 >= lo + 5) & (b1 <= hi - 5), axis=1)
        n_fixed += int(fixed[inner][core].sum())
        n_inside += sum(inside_at(pose1)(i, j, k) for i in range(c[0] - 1, c[0] + 4)
                        for j in range(c[1] - 1, c[1] + 4) for k in range(c[2] - 1, c[2] + 4))
        u2, v2, C2, F2 = L.g2p(u1[core], F1[core], fixed[inner][core], V1, lo)
        got = ids[inner][core]
        gu = S2["u"][:, torch.from_numpy(got).cuda()].T.double().cpu().numpy()
        gF = S2["Fm"][:, torch.from_numpy(got).cuda()].T.double().cpu().numpy().reshape(-1, 3, 3)
        du = max(du, float(np.abs(gu - u2).max()))
        dF = max(dF, float(np.abs(gF - (F2 - np.eye(3))).max()))
        sF = max(sF, float(np.abs(F2 - np.eye(3)).max()))
        nck += len(got)
    assert nck >= 8 * 100
    assert n_inside > 0 and n_fixed > 0  # both boundary conditions act in the checked stencils
    assert sMG > 0 and dMG / sMG <= 1e-5, (dMG, sMG)
    assert dM / sM <= 1e-5, (dM, sM)
    assert du <= 1e-4, du
    assert sF > 1e-3 and dF <= 1e-4 * sF, (dF, sF)

    # the benchmark's frame of that state, 640 x 480 over the top face: the
    # height map against the oracle's from the same positions (Sec. III-B),
    # and the image against the oracle's shading of the same height map
    # (Eqs. 12-14)
    win = W.top_window(b)
    Lt = W.default_lights()
    Hd = torch.empty((480, 640), device="cuda")
    img = g.render(640, 480, win, rp=T.render_params_from(Lt), out_height=Hd)
    o = oracle.Sim(b.nx, b.ny, b.nz, dx, b.E, b.nu, b.rho, b.pad_side, b.pad_bottom, b.pad_top)
    u0, fl = oracle.lattice(b.nx, b.ny, b.nz, b.pad_side, b.pad_bottom, b.seed)
    o.set_rest(u0)
    o.set_state(S2["u"].cpu().numpy(), flags=S2["flags"].cpu().numpy())
    Hg = Hd.cpu().numpy().astype(np.float64)
    Ho = o.heightmap(win, 640, 480)
    assert Ho.min() < g.z_top - 0.3e-3  # the press shows
    assert np.abs(Hg - Ho).max() <= 1e-3 * dx
    rpo = oracle.render_params(Lt["n_lights"], Lt["dirs"], Lt["diffuse"], Lt["specular"], Lt["ambient"],
                               Lt["ka"], Lt["kd"], Lt["ks"], Lt["alpha"])
    Io = oracle.shade(Hg, (win[2] - win[0]) / 640, (win[3] - win[1]) / 480, g.z_top, rpo)
    assert np.abs(img.cpu().numpy() - Io).max() <= 2e-5
