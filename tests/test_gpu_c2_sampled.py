"""Parity at the full batched workload in the launch configuration the
benchmark times (256 uneven sensors, 56.3 M particles in one handle, 8 x 8 x 4
sort blocks, the fused transfer), on outputs the oracle's per-particle
routines can compute one by one.

Every sensor is pressed for 200 substeps; the state of a few sensors is read
back, two more substeps run on the GPU for the whole batch, and around a
sampled node of each of those sensors the two substeps are recomputed in FP64
from the read-back state (oracle/local.py: P2G, grid velocity, G2P,
F update and advection, twice).  Compared: position and F of every particle
whose stencil the box covers, after the closing G2P (1e-4 cells; F - I to 1e-4
of its largest entry).  The sensors are the thick ones (12 cells or more)
pressed by a sphere, and the node sits two millimetres outside the sphere's
radius, clear of the fixed base and the padding band, so that no boundary
condition acts inside the box."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.local import Local, velocity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def test_c2_two_substeps_at_sampled_particles():
    import paper_2301_08343_gb300 as T
    import oracle
    specs = W.c2_instances(256, seed_base=1000)
    bt = T.TacchiBatch([b for b, _ in specs])
    assert bt.N_total > 50_000_000
    K = T.IndenterKind
    kinds = {"sphere": K.SPHERE, "cylinder": K.CYLINDER, "cone": K.CONE, "prism": K.PRISM}
    n, dt = 200, W.C2_DT
    for i, (b, ind) in enumerate(specs):
        bt.set_indenter(i, kinds[ind["kind"]], ind["params"], ind["pose"], (0, 0, -ind["depth"] / (n * dt), 0, 0, 0))
    bt.step(n, dt)
    picks = [i for i, (b, ind) in enumerate(specs) if ind["kind"] == "sphere" and b.nz >= 12][:3]
    assert len(picks) == 3
    S = {i: bt.get_state(i) for i in picks}
    poses = {i: bt.indenter_pose(i) for i in picks}
    bt.step(2, dt)
    S2 = {i: bt.get_state(i) for i in picks}
    assert bt.status() == 0
    du, dF, sF, nck = 0.0, 0.0, 0.0, 0
    for i in picks:
        b, ind = specs[i]
        dx = b.dx
        L = Local(dx, dt, b.E, b.nu, b.rho)
        org = np.array([-b.pad_side * dx, -b.pad_side * dx, -b.pad_bottom * dx])
        cc = (np.array(poses[i][:3]) - org) / dx             # sphere centre (cells)
        R = ind["params"][0] / dx
        # the node nearest the sphere whose box lies inside the sensor's sides
        # and whose 11-node velocity neighbourhood stays clear of the sphere,
        # at a depth clear of the base
        cz = b.pad_bottom + 7 + min(3, b.nz - 12)
        best = None
        for cx in range(b.pad_side + 6, b.pad_side + b.nx - 6):
            for cy in range(b.pad_side + 6, b.pad_side + b.ny - 6):
                dist = math.sqrt((cx - cc[0]) ** 2 + (cy - cc[1]) ** 2 + (cz - cc[2]) ** 2) - R
                if dist > 6 * math.sqrt(3) + 2 and (best is None or dist < best[0]):
                    best = (dist, cx, cy)
        assert best is not None
        c = np.array([best[1], best[2], cz])
        lo, hi = c - 6, c + 6
        u = S[i]["u"]
        base = torch.floor(u - 0.5).to(torch.int32)
        sel = ((base[0] >= lo[0]) & (base[0] <= hi[0]) & (base[1] >= lo[1]) & (base[1] <= hi[1]) &
               (base[2] >= lo[2]) & (base[2] <= hi[2])).nonzero().flatten()
        ids = sel.cpu().numpy()
        up = u[:, sel].T.double().cpu().numpy()
        vp = S[i]["v"][:, sel].T.double().cpu().numpy()
        Cp = S[i]["C"][:, sel].T.double().cpu().numpy().reshape(-1, 3, 3)
        Fp = S[i]["Fm"][:, sel].T.double().cpu().numpy().reshape(-1, 3, 3) + np.eye(3)
        fixed = (S[i]["flags"][sel].cpu().numpy() & 1) > 0
        assert len(ids) > 1000 and not fixed.any()
        shape = tuple((hi - lo + 3)[::-1])
        M0, MG0 = L.p2g(up, vp, Cp, Fp, lo, shape)
        bp = np.floor(up - 0.5).astype(int)
        inner = np.all((bp >= lo + 2) & (bp <= hi - 2), axis=1)
        u1, v1, C1, F1 = L.g2p(up[inner], Fp[inner], fixed[inner], velocity(M0, MG0), lo)
        M1, MG1 = L.p2g(u1, v1, C1, F1, lo, shape)
        b1 = np.floor(u1 - 0.5).astype(int)
        core = np.all((b1 >= lo + 5) & (b1 <= hi - 5), axis=1)
        u2, _, _, F2 = L.g2p(u1[core], F1[core], fixed[inner][core], velocity(M1, MG1), lo)
        got = torch.from_numpy(ids[inner][core]).cuda()
        gu = S2[i]["u"][:, got].T.double().cpu().numpy()
        gF = S2[i]["Fm"][:, got].T.double().cpu().numpy().reshape(-1, 3, 3)
        du = max(du, float(np.abs(gu - u2).max()))
        dF = max(dF, float(np.abs(gF - (F2 - np.eye(3))).max()))
        sF = max(sF, float(np.abs(F2 - np.eye(3)).max()))
        nck += len(got)
    assert nck >= 3 * 50
    assert du <= 1e-4, du
    assert sF > 1e-5 and dF <= 1e-4 * sF + 2e-7, (dF, sF)
