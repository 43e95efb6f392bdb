"""C-ABI checks that need no GPU: the library builds, loads and exports every
symbol declared in include/*.h; host-only entry points behave; argument
validation happens before any CUDA call."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2301_08343_gb300 import build
    build.build()
    from paper_2301_08343_gb300 import _lib
    return _lib.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(tacchi_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "tacchi_create" in names and "tacchi_step" in names and "tacchi_render" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_declares_every_header_function(L):
    from paper_2301_08343_gb300 import _lib
    bound = set(_lib.SIGNATURES) | set(_lib.EXTRA_SIGNATURES)
    assert set(declared_functions()) <= bound


def test_host_lattice_is_bit_identical_to_the_oracle(L):
    import paper_2301_08343_gb300 as T
    for (nx, ny, nz, seed, jit) in [(5, 4, 3, 0, True), (24, 24, 6, 0, True), (3, 2, 2, 99, False)]:
        u, fl = T.init_lattice(nx, ny, nz, 4, 3, seed, jit)
        uo, flo = oracle.lattice(nx, ny, nz, 4, 3, seed, jit)
        assert np.array_equal(u.view(np.uint32), uo.view(np.uint32))
        assert np.array_equal(fl, flo)


def test_status_strings_and_version(L):
    for s in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert L.tacchi_status_string(s)
    assert L.tacchi_status_string(-99) == b"unknown status"
    assert L.tacchi_version() >= 100


def _desc(**kw):
    from paper_2301_08343_gb300 import _lib
    d = _lib.ElastomerDesc()
    vals = dict(extent=(6e-3, 6e-3, 2e-3), dx=0.5e-3, E=3e5, nu=0.45, rho=1000.0)
    vals.update(kw)
    for a in range(3):
        d.extent_m[a] = vals["extent"][a]
    d.dx_m, d.E_pa, d.nu, d.density = vals["dx"], vals["E"], vals["nu"], vals["rho"]
    for k in ("pad_side", "pad_bottom", "pad_top"):
        if k in kw:
            setattr(d, k, kw[k])
    if "block" in kw:
        for a in range(3):
            d.block[a] = kw["block"][a]
    if "tpc" in kw:
        d.threads_per_cell = kw["tpc"]
    return d


@pytest.mark.parametrize("bad", [
    dict(dx=0.0), dict(dx=-1.0), dict(E=0.0), dict(nu=0.5), dict(nu=-1.0), dict(rho=0.0),
    dict(extent=(6.1e-3, 6e-3, 2e-3)), dict(extent=(0.0, 6e-3, 2e-3)), dict(pad_side=2),
    dict(pad_top=1), dict(block=(3, 3, 3)), dict(extent=(float("nan"), 6e-3, 2e-3)),
    dict(block=(8, 8, 8), tpc=3), dict(tpc=2), dict(block=(16, 8, 4), tpc=3),
    dict(pad_side=1025), dict(extent=(0.725, 0.725, 0.5e-3), pad_top=1024),  # 2.19e9 grid nodes
])
def test_create_rejects_invalid_descriptions_before_touching_cuda(L, bad):
    d = _desc(**bad)
    h = C.c_void_p()
    assert L.tacchi_create(C.byref(d), None, C.byref(h)) == -1
    assert not h.value


def test_null_arguments_are_rejected(L):
    assert L.tacchi_create(None, None, None) == -1
    assert L.tacchi_step(None, 1, 1e-5) == -1
    assert L.tacchi_sync(None) == -1
    assert L.tacchi_get_state(None, None, None, None, None, None) == -1
    assert L.tacchi_init_lattice(0, 1, 1, 4, 3, 0, 1, None, None) == -1
    from paper_2301_08343_gb300 import _lib
    rp = _lib.RenderParams()
    rp.n_lights = 9
    assert L.tacchi_shade(C.byref(rp), C.c_void_p(16), 4, 4, 1e-4, 1e-4, 0.0, C.c_void_p(16), None) == -1


def test_null_handles_of_the_later_entry_points_are_rejected(L):
    # the particle indenter, markers, penetration map and comparison renderer
    # check their handle and arguments before any CUDA call
    from paper_2301_08343_gb300 import _lib
    rp = _lib.RenderParams()
    win = (C.c_double * 4)(0.0, 0.0, 1e-3, 1e-3)
    buf = C.c_void_p(16)
    assert L.tacchi_batch_render_smoothed(None, 0, C.byref(rp), 8, 8, win, 1e-4, buf, buf) == -1
    assert L.tacchi_render_smoothed(None, C.byref(rp), 8, 8, win, 1e-4, buf, buf) == -1
    assert L.tacchi_batch_penetration_map(None, 0, 8, 8, win, buf) == -1
    assert L.tacchi_batch_markers(None, 0, 4, buf, buf) == -1
    assert L.tacchi_set_indenter_particles(None, 4, None, 1e-6) == -1
