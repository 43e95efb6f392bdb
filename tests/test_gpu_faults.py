"""Failure detection without a GPU fault: invalid inputs are refused on the
host, or turned by the kernels' own checks into a status that the next
synchronising call returns, and the handle keeps working afterwards.

  * a non-positive or non-finite substep, a height map holding NaN, a
    tilted pose for the penetration map: INVALID_ARG before any launch;
  * an indenter posed far outside the grid: no effect, status 0;
  * a velocity field that carries particles several cells in one substep
    (a CFL violation): the transfer scatters nothing out of its tile and
    reports an error instead; after set_state the handle steps cleanly."""
import math

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


def sensor():
    import paper_2301_08343_gb300 as T
    b = W.Block(8, 8, 4, 0.5e-3, seed=6)
    return T, b, T.Tacchi(b.extent_m, b.dx, b.E, b.nu, b.rho, seed=b.seed)


def test_invalid_arguments_are_refused_on_the_host():
    from paper_2301_08343_gb300 import _lib
    T, b, g = sensor()
    L = _lib.lib()
    for dt in (0.0, -1e-5, float("nan"), float("inf")):
        assert L.tacchi_step(g._h, 1, dt) == -1
    assert L.tacchi_step(g._h, 0, 1e-5) == -1
    hm = np.zeros((8, 8), np.float32)
    hm[3, 4] = np.nan
    with pytest.raises(RuntimeError):
        g.set_indenter(T.IndenterKind.HEIGHTMAP, (1e-3,), (2e-3, 2e-3, 3e-3, 1, 0, 0, 0), (0,) * 6,
                       hm=hm, hm_pixel=0.1e-3)
    bt = T.TacchiBatch([b])
    tilt = (2e-3, 2e-3, 3e-3, math.cos(0.2), math.sin(0.2), 0.0, 0.0)
    bt.set_indenter(0, T.IndenterKind.SPHERE, (2e-3,), tilt, (0,) * 6)
    with pytest.raises(RuntimeError):
        bt.penetration_map(0, 16, 16, W.top_window(b))
    assert g.status() == 0 and bt.status() == 0


def test_indenter_far_outside_the_grid_has_no_effect():
    T, b, g = sensor()
    u0 = g.get_state()["u"].clone()
    g.set_indenter(T.IndenterKind.SPHERE, (2e-3,), (1.0, -2.0, 5.0, 1, 0, 0, 0), (0, 0, -1.0, 0, 0, 0))
    g.step(50, 1e-5)
    s = g.get_state()
    assert s["status"] == 0
    assert torch.equal(s["u"], u0)


def test_cfl_violation_is_reported_and_the_handle_recovers():
    T, b, g = sensor()
    st = g.get_state()
    u0 = st["u"].clone()
    # 60 m/s at dt = 1e-5 s and dx = 0.5 mm: 1.2 cells in one substep (the
    # particles stay inside the grid's padding, so no other error is raised)
    v = torch.zeros_like(u0)
    v[0] = 60.0
    g.set_state(u0, v)
    g.step(1, 1e-5)
    assert g.status() == -8  # TACCHI_ERR_CFL
    g.set_state(u0)
    g.step(20, 1e-5)
    s = g.get_state()
    assert s["status"] == 0
    assert torch.equal(s["u"], u0)
