"""The pipelined fused transfer (a persistent grid over the sort's block
records, bulk copies of the next block's slots, home cells and grid velocities
while a block's particles run) against the per-block transfer kernel.

Both run the same particle loop in the same cell order, so their states differ
only by the order in which cells' node sums reach the grid (vector reductions
to global memory from CTAs running at different times): within the bounds of
reordered FP32 sums."""
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


def c0_sensor(pipelined):
    import paper_2301_08343_gb300 as T
    b = W.C0
    g = T.Tacchi(b.extent_m, b.dx, b.E, b.nu, b.rho, seed=b.seed, pad_side=b.pad_side,
                 pad_bottom=b.pad_bottom, pad_top=b.pad_top)
    g.set_pipeline(pipelined)
    g.set_indenter(T.IndenterKind.SPHERE, (W.C0_SPHERE_R,), W.c0_sphere_pose(), W.c0_sphere_vel())
    return T, g


def test_pipeline_switch_and_its_plan():
    _, g = c0_sensor(False)
    assert g.block == (8, 8, 4) and g.threads_per_cell == 1
    assert not g.pipelined  # the per-block kernel is the default
    g.set_pipeline(True)
    assert g.pipelined
    g.set_transfer((4, 4, 4), 1)  # no pipelined form: the per-block kernel runs
    assert not g.pipelined
    g.set_transfer((8, 8, 4), 1)
    assert g.pipelined
    g.set_launch(True)  # the persistent step has its own transfer
    assert not g.pipelined


def test_pipelined_press_matches_the_per_block_kernel():
    _, a = c0_sensor(False)
    _, p = c0_sensor(True)
    for _ in range(3):
        a.step(100, W.C0_DT)
        p.step(100, W.C0_DT)
    sa, sp = a.get_state(), p.get_state()
    assert sa["status"] == 0 and sp["status"] == 0
    assert np.abs(sa["u"].cpu().numpy() - sp["u"].cpu().numpy()).max() <= 1e-5
    assert np.abs(sa["Fm"].cpu().numpy() - sp["Fm"].cpu().numpy()).max() <= 1e-5
    win = W.top_window(W.C0)
    ha = a.heightmap(120, 120, win).cpu().numpy()
    hp = p.heightmap(120, 120, win).cpu().numpy()
    assert np.abs(ha - hp).max() <= 1e-3 * W.C0.dx


def test_pipelined_step_follows_the_sorts():
    """A drifting block: its particles cross sort blocks every few substeps,
    so the block records and home cells are rebuilt by the sort between
    pipelined transfers."""
    import paper_2301_08343_gb300 as T
    b = W.Block(24, 16, 6, 0.5e-3, seed=3, pad_side=12)
    out = []
    for pipelined in (False, True):
        g = T.Tacchi(b.extent_m, b.dx, b.E, b.nu, b.rho, seed=b.seed, pad_side=b.pad_side, fix_base=False)
        g.set_pipeline(pipelined)
        u0 = g.get_state()["u"].clone()
        v = torch.zeros_like(u0)
        v[0], v[1] = 3.0, -1.5  # 0.06 and 0.03 cells per substep
        g.set_state(u0, v)
        g.profile(reset=True)
        g.step(60, 1e-5)
        s = g.get_state()
        assert s["status"] == 0
        out.append((s["u"].cpu().numpy(), g.profile()["sort_runs"]))
    (ua, na), (up, np_) = out
    assert na > 0 and np_ > 0
    assert np.abs(ua - up).max() <= 1e-5


def test_pipelined_batch_matches_the_per_block_kernel():
    import paper_2301_08343_gb300 as T
    specs = W.c2_instances(6, seed_base=1000)
    K = T.IndenterKind
    kinds = {"sphere": K.SPHERE, "cylinder": K.CYLINDER, "cone": K.CONE, "prism": K.PRISM}
    out = []
    for pipelined in (False, True):
        bt = T.TacchiBatch([b for b, _ in specs])
        bt.set_pipeline(pipelined)
        assert bt.pipelined == pipelined
        for i, (b, ind) in enumerate(specs):
            bt.set_indenter(i, kinds[ind["kind"]], ind["params"], ind["pose"],
                            (0, 0, -ind["depth"] / (200 * W.C2_DT), 0, 0, 0))
        bt.step(200, W.C2_DT)
        assert bt.status() == 0
        out.append([bt.get_state(i)["u"].cpu().numpy() for i in range(len(specs))])
    for a, p in zip(*out):
        assert np.abs(a - p).max() <= 1e-4  # 200 substeps of reordered FP32 reductions


def test_pipelined_copy_wait_is_bounded_and_the_handle_recovers():
    """Every copy wait is told to wait for an arrival that never comes: each
    CTA gives up, supplies the missing arrival itself, waits for its copies
    in flight and leaves; the step reports TACCHI_ERR_TIMEOUT and the handle
    steps normally once the wait is restored."""
    import math
    from paper_2301_08343_gb300 import _lib
    _, g = c0_sensor(True)
    u0 = g.get_state()["u"].clone()
    with pytest.raises(_lib.TacchiError):
        g.set_barrier_wait(1 << 24, extra_arrivals=70000)
    g.set_barrier_wait(1 << 14, extra_arrivals=1)
    g.step(5, W.C0_DT)
    assert g.status() == -6  # TACCHI_ERR_TIMEOUT
    g.set_barrier_wait(1 << 24, extra_arrivals=0)
    g.set_state(u0)
    g.step(5, W.C0_DT)
    s = g.get_state()
    assert s["status"] == 0
    assert math.isfinite(float(s["u"].abs().max()))



def test_block_beyond_the_grouping_capacity():
    """4,000 particles packed into one 8 x 8 x 4 block (capacity 3,072): that
    block takes the ungrouped path, one particle per thread with its own
    scatter, in both kernels (the pipelined one then copies no slots or home
    cells for it); the step reports no error and the two agree."""
    out = []
    for pipelined in (False, True):
        _, g = c0_sensor(pipelined)
        g.set_indenter(vel=(0, 0, 0, 0, 0, 0))
        u = g.get_state()["u"].clone()
        rng = np.random.default_rng(4)
        k = 4000
        b0 = np.array([8.0, 8.0, 4.0])
        ext = np.array([8.0, 8.0, 4.0])
        # home cells floor(u - 1/2) inside the block [b0, b0 + ext)
        pts = b0 + 0.5 + rng.random((k, 3)) * ext
        u[:, :k] = torch.as_tensor(pts.T, dtype=torch.float32, device=u.device)
        g.set_state(u)
        g.step(5, W.C0_DT)
        s = g.get_state()
        assert s["status"] == 0
        out.append(s["u"].cpu().numpy())
    assert np.abs(out[0] - out[1]).max() <= 1e-5


def test_single_handle_autotune_keeps_the_state_and_reports_its_plan():
    _, g = c0_sensor(False)
    g.step(10, W.C0_DT)
    before = g.get_state()["u"].clone()
    best, ms = g.autotune(8, W.C0_DT)
    assert best in [(4, 4, 4, 1), (8, 8, 4, 1), (8, 8, 8, 1), (16, 8, 4, 1), (8, 8, 4, 3), (4, 4, 4, 3)]
    assert g.block == tuple(best[:3]) and g.threads_per_cell == best[3]
    assert len(ms) == 6 and all(v > 0 for v in ms.values())
    assert torch.equal(g.get_state()["u"], before)
    g.step(10, W.C0_DT)
    assert g.get_state()["status"] == 0
