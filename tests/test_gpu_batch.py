"""Batched sensors (many instances in one handle) against single-instance
runs and the oracle (GPU, through the C ABI).

Tolerance: a batched instance and the same instance run alone differ only by
the order of FP32 reductions, so positions agree to 1e-4 cells after 60
substeps; against the FP64 oracle, 1e-3 cells (as for single instances)."""
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


def T():
    import paper_2301_08343_gb300 as T_
    return T_


BLOCKS = [W.Block(6, 5, 2, 0.5e-3, seed=11), W.Block(9, 7, 3, 0.5e-3, seed=12),
          W.Block(4, 4, 2, 0.5e-3, seed=13), W.Block(12, 10, 4, 0.5e-3, seed=14)]


def indenter(i, b):
    R = [1.2e-3, 1.5e-3, 1.0e-3, 2.0e-3][i]
    yaw = 0.3 * i
    pose = (b.nx * b.dx / 2 + 0.1e-3 * i, b.ny * b.dx / 2, b.nz * b.dx + R - 0.05e-3,
            math.cos(yaw / 2), 0.0, 0.0, math.sin(yaw / 2))
    vel = (0.01 * i, 0.0, -0.2, 0.0, 0.0, 0.5 * i)
    if i % 2 == 0:
        return "sphere", (R,), pose, vel
    return "cylinder", (R, 1.5e-3), pose, vel


def kind(name):
    K = T().IndenterKind
    return {"sphere": K.SPHERE, "cylinder": K.CYLINDER}[name]


def okind(name):
    return {"sphere": oracle.IND_SPHERE, "cylinder": oracle.IND_CYLINDER}[name]


def run_batch(n=60, dt=1e-5, shape=None):
    bt = T().TacchiBatch(BLOCKS, sort_block=shape)
    for i, b in enumerate(BLOCKS):
        name, params, pose, vel = indenter(i, b)
        bt.set_indenter(i, kind(name), params, pose, vel)
    bt.step(n, dt)
    assert bt.status() == 0
    return bt


def test_batched_instances_match_single_instance_runs_and_oracle():
    n, dt = 60, 1e-5
    bt = run_batch(n, dt)
    for i, b in enumerate(BLOCKS):
        name, params, pose, vel = indenter(i, b)
        g = T().Tacchi(b.extent_m, b.dx, b.E, b.nu, b.rho, seed=b.seed, pad_side=b.pad_side,
                       pad_bottom=b.pad_bottom, pad_top=b.pad_top)
        g.set_indenter(kind(name), params, pose, vel)
        g.step(n, dt)
        sb = bt.get_state(i)
        sg = g.get_state()
        assert sb["status"] == 0 and sg["status"] == 0
        ub, ug = sb["u"].cpu().numpy(), sg["u"].cpu().numpy()
        assert np.abs(ub - ug).max() <= 1e-4
        assert np.allclose(bt.indenter_pose(i), g.indenter_pose(), rtol=0, atol=1e-15)
        win = W.top_window(b)
        hb = bt.heightmap(i, 40, 30, win).cpu().numpy()
        hg = g.heightmap(40, 30, win).cpu().numpy()
        assert np.abs(hb - hg).max() <= 1e-3 * b.dx
        if i == 1:
            o = oracle.Sim(b.nx, b.ny, b.nz, b.dx, b.E, b.nu, b.rho, b.pad_side, b.pad_bottom, b.pad_top)
            u0, fl = oracle.lattice(b.nx, b.ny, b.nz, b.pad_side, b.pad_bottom, b.seed)
            o.set_state(u0, flags=fl)
            o.set_indenter(okind(name), params, pose, vel)
            assert o.run(n, dt) == 0
            assert np.abs(ub - o.state()[0]).max() <= 1e-3


@pytest.mark.parametrize("shape", [(4, 4, 4, 1), (8, 8, 4, 1), (8, 8, 8, 1), (16, 8, 4, 1), (8, 8, 4, 3),
                                   (4, 4, 4, 3)])
def test_every_transfer_plan_gives_the_same_batch(shape):
    """Every block shape, with one thread per cell or three, steps the batch
    alike (FP32 summation order only)."""
    ref = run_batch(shape=(4, 4, 4, 1))
    assert ref.transfer_plan() == ((4, 4, 4), 1)
    got = run_batch(shape=shape)
    assert got.transfer_plan() == (tuple(shape[:3]), shape[3])
    for i in range(len(BLOCKS)):
        a = ref.get_state(i)["u"].cpu().numpy()
        b = got.get_state(i)["u"].cpu().numpy()
        assert np.abs(a - b).max() <= 1e-4


def test_autotune_keeps_the_state_and_picks_a_supported_shape():
    bt = T().TacchiBatch(BLOCKS)
    for i, b in enumerate(BLOCKS):
        name, params, pose, vel = indenter(i, b)
        bt.set_indenter(i, kind(name), params, pose, vel)
    bt.step(10, 1e-5)
    before = [bt.get_state(i)["u"].clone() for i in range(len(BLOCKS))]
    poses = [bt.indenter_pose(i) for i in range(len(BLOCKS))]
    best, ms = bt.autotune(8, 1e-5)
    assert best in [(4, 4, 4, 1), (8, 8, 4, 1), (8, 8, 8, 1), (16, 8, 4, 1), (8, 8, 4, 3), (4, 4, 4, 3)]
    assert bt.transfer_plan() == (best[:3], best[3])
    assert len(ms) == 6 and all(v > 0 for v in ms.values())
    for i in range(len(BLOCKS)):
        assert torch.equal(bt.get_state(i)["u"], before[i])
        assert bt.indenter_pose(i) == poses[i]
    bt.step(50, 1e-5)
    ref = run_batch(60, 1e-5)
    for i in range(len(BLOCKS)):
        assert np.abs(bt.get_state(i)["u"].cpu().numpy() - ref.get_state(i)["u"].cpu().numpy()).max() <= 1e-4


def test_batch_instance_index_is_checked():
    bt = T().TacchiBatch(BLOCKS[:2])
    from paper_2301_08343_gb300 import _lib
    import ctypes as C
    p = (C.c_double * 7)()
    assert _lib.lib().tacchi_batch_get_indenter_pose(bt._h, 2, p) == -1
    assert _lib.lib().tacchi_batch_get_indenter_pose(bt._h, -1, p) == -1
    n = C.c_int()
    assert _lib.lib().tacchi_batch_size(bt._h, C.byref(n)) == 0 and n.value == 2
