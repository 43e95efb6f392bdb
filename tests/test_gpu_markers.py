"""Marker motion (the outlook of the paper's Sec. V): a marker follows the
top-layer particle whose rest sub-cell contains it (GPU, through the C ABI).

Checks: a rigid translation of every particle moves every marker by exactly
that translation; after a press, each marker's displacement equals the
displacement of the particle the host selects by the documented rule from
the state (rest position in the marker's dx/2 sub-cell, top layer), and a
marker at a pixel centre agrees bit for bit with the displacement map."""
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


def make():
    import paper_2301_08343_gb300 as T
    b = W.Block(10, 8, 3, 0.5e-3, seed=21)
    return T, b, T.Tacchi(b.extent_m, b.dx, b.E, b.nu, b.rho, seed=b.seed)


def test_translation_moves_markers_exactly():
    T, b, g = make()
    u0 = g.get_state()["u"].clone()
    shift = torch.tensor([0.25, -0.125, 0.0625], device=u0.device).reshape(3, 1)  # cells, exact in FP32
    g.set_state(u0 + shift)
    rng = np.random.default_rng(0)
    xy = rng.uniform([0, 0], [b.nx * b.dx, b.ny * b.dx], (500, 2)).astype(np.float32)
    d = g.markers(xy).cpu().numpy()
    assert np.allclose(d, shift.cpu().numpy().ravel() * b.dx, rtol=0, atol=1e-9)


def test_markers_follow_their_particles_after_a_press():
    T, b, g = make()
    st0 = g.get_state()
    u0 = st0["u"].cpu().numpy().astype(np.float64)
    top = (st0["flags"].cpu().numpy() & 2) > 0
    R = 2e-3
    g.set_indenter(T.IndenterKind.SPHERE, (R,), (b.nx * b.dx / 2, b.ny * b.dx / 2, b.nz * b.dx + R - 0.05e-3, 1, 0, 0, 0),
                   (0, 0, -0.2, 0, 0, 0))
    g.step(120, 1e-5)
    u = g.get_state()["u"].cpu().numpy().astype(np.float64)
    org = np.array(g.origin)
    rest_xy = u0[:2, top].T * b.dx + org[:2]
    ids = np.nonzero(top)[0]
    rng = np.random.default_rng(1)
    xy = rng.uniform([0, 0], [b.nx * b.dx, b.ny * b.dx], (400, 2)).astype(np.float32)
    d = g.markers(xy).cpu().numpy()
    half = np.float32(0.5) * np.float32(b.dx)
    for k in range(len(xy)):
        i = int(np.clip(np.floor(np.float32(xy[k, 0]) / half), 0, 2 * b.nx - 1))
        j = int(np.clip(np.floor(np.float32(xy[k, 1]) / half), 0, 2 * b.ny - 1))
        inside = ((np.floor(rest_xy[:, 0] / (0.5 * b.dx)) == i) & (np.floor(rest_xy[:, 1] / (0.5 * b.dx)) == j))
        assert inside.sum() == 1
        p = ids[inside][0]
        expect = (u[:, p] - u0[:, p]) * b.dx
        assert np.allclose(d[k], expect, rtol=0, atol=2e-9), (k, d[k], expect)
    # a marker at a pixel centre reads what the displacement map reads there
    # (16 x 16 pixels over 10 x 8 cells: no pixel centre on a sub-cell edge)
    bt = T.TacchiBatch([b])
    bt.set_indenter(0, T.IndenterKind.SPHERE, (R,), (b.nx * b.dx / 2, b.ny * b.dx / 2, b.nz * b.dx + R - 0.05e-3, 1, 0, 0, 0),
                    (0, 0, -0.2, 0, 0, 0))
    bt.step(60, 1e-5)
    win = (0.0, 0.0, b.nx * b.dx, b.ny * b.dx)
    dm = bt.displacement_map(0, 16, 16, win)
    cx = (np.arange(16) + 0.5) * (b.nx * b.dx / 16)
    cy = (np.arange(16) + 0.5) * (b.ny * b.dx / 16)
    X, Y = np.meshgrid(cx, cy)
    pts = np.stack([X.ravel(), Y.ravel()], 1).astype(np.float32)
    dk = bt.markers(0, pts).reshape(16, 16, 3)
    assert float(dm.abs().max()) > 1e-6
    assert torch.equal(dk, dm)
