"""tacchi_heightmap_static against tacchi_heightmap (GPU, through the C ABI).

Callers that cannot allocate device memory while they run, such as a robot
simulator's real-time control thread or a plugin whose host application owns
the device-memory budget, use tacchi_heightmap_static.  Its only scratch is a
static device array, so it must give the same height map as the allocating
entry point, call after call, although every call reuses that array.  The
tolerance is the one the other height-map tests use: 1e-3 dx.

This file is named so that pytest collects it last.
"""
import ctypes as C

import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_static_heightmap_matches_the_allocating_entry_point_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_08343_gb300 as T
    from paper_2301_08343_gb300 import _lib

    b = W.C0
    sim = T.Tacchi(b.extent_m, b.dx, b.E, b.nu, b.rho, seed=b.seed, pad_side=b.pad_side,
                   pad_bottom=b.pad_bottom, pad_top=b.pad_top)
    rest = sim.get_state()
    assert rest["status"] == 0
    surf = torch.nonzero(rest["flags"] & 2).flatten().to(torch.int32).contiguous()
    z0 = rest["u"][2, surf.long()].contiguous()
    sim.set_indenter(T.IndenterKind.SPHERE, (W.C0_SPHERE_R,), W.c0_sphere_pose(), W.c0_sphere_vel())
    L = _lib.lib()
    origin = (C.c_double * 2)(*sim.origin[:2])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    calls = [(150, 120, 120, W.top_window(b), 8),
             (200, 97, 83, (-1.5e-3, -1e-3, 13.5e-3, 12.5e-3), 5)]
    for n, w, h, win, fill in calls:
        sim.step(n, W.C0_DT)
        ref = sim.heightmap(w, h, win, fill_radius=fill)
        st = sim.get_state()
        assert st["status"] == 0
        out = torch.full((h, w), float("nan"), device="cuda")
        rc = L.tacchi_heightmap_static(_lib.ptr(st["u"]), sim.N, _lib.ptr(surf), _lib.ptr(z0),
                                       surf.numel(), b.dx, origin, sim.z_top, w, h,
                                       (C.c_double * 4)(*win), fill, _lib.ptr(out), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert bool(torch.isfinite(out).all())
        assert (out - ref).abs().max().item() <= 1e-3 * b.dx

    # a map larger than the static scratch is refused before any launch
    big = torch.empty((1024, 1025), device="cuda")
    rc = L.tacchi_heightmap_static(_lib.ptr(st["u"]), sim.N, _lib.ptr(surf), _lib.ptr(z0),
                                   surf.numel(), b.dx, origin, sim.z_top, 1025, 1024,
                                   (C.c_double * 4)(*W.top_window(b)), 8, _lib.ptr(big), stream)
    assert rc == -1
