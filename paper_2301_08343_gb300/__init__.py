"""GB300-native Tacchi: MLS-MPM elastomer simulation and tactile rendering.

Thin Python binding of the C ABI in ``include/tacchi.h``.  PyTorch provides
device memory and streams; every step of the simulation and rendering runs in
the library's CUDA kernels (``libtacchi.so``).  There is no CPU fallback: the
binding raises when the library or a CUDA device is missing.

Method: Tacchi (arXiv 2301.08343) -- Sec. III-A (MPM substep, Eqs. 1-11),
Sec. III-B (height map and Phong shading, Eqs. 12-14), Sec. III-C (the
indenter pose/velocity supplied by a main simulator).
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import _lib
from ._lib import TacchiError, check, lib, ptr

__all__ = ["Tacchi", "TacchiError", "IndenterKind", "default_render_params", "shade",
           "init_lattice", "lib"]


# Transfer plans in the autotuner's order: sort block / threads per cell.
TRANSFER_PLANS = ("4x4x4/1", "8x8x4/1", "8x8x8/1", "16x8x4/1", "8x8x4/3", "4x4x4/3")


class Contact:
    STICKY, SLIP = 0, 1


class IndenterKind:
    NONE, SPHERE, CYLINDER, CONE, PRISM, HEIGHTMAP = range(6)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("paper_2301_08343_gb300 needs a CUDA device (no CPU fallback)")
    return torch


def _stream_handle(torch, stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def default_render_params(n_lights=3, elevation_deg=30.0, ka=0.2, kd=0.6, ks=0.2, alpha=5.0):
    """Three RGB lights 120 degrees apart in azimuth on the camera side
    (this project's defaults; Eq. 12 leaves the constants to calibration)."""
    rp = _lib.RenderParams()
    rp.n_lights = n_lights
    el = math.radians(elevation_deg)
    cols = [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)]
    for m in range(n_lights):
        az = math.radians(90.0 + 120.0 * m)
        d = (math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), -math.sin(el))
        for a in range(3):
            rp.dir[m][a] = d[a]
            rp.diffuse[m][a] = cols[m % 3][a]
            rp.specular[m][a] = 1.0
    for a in range(3):
        rp.ambient[a] = 1.0
    rp.ka, rp.kd, rp.ks, rp.alpha = ka, kd, ks, alpha
    return rp


def render_params_from(d):
    """RenderParams from a dict with n_lights, dirs, diffuse, specular,
    ambient, ka, kd, ks, alpha."""
    rp = _lib.RenderParams()
    rp.n_lights = d["n_lights"]
    for m in range(d["n_lights"]):
        for a in range(3):
            rp.dir[m][a] = d["dirs"][m][a]
            rp.diffuse[m][a] = d["diffuse"][m][a]
            rp.specular[m][a] = d["specular"][m][a]
    for a in range(3):
        rp.ambient[a] = d["ambient"][a]
    rp.ka, rp.kd, rp.ks, rp.alpha = d["ka"], d["kd"], d["ks"], d["alpha"]
    return rp


def init_lattice(nx, ny, nz, pad_side=4, pad_bottom=3, seed=0, jitter=True):
    """Host copy of the particle lattice tacchi_create makes (no GPU)."""
    n = 8 * nx * ny * nz
    u = np.zeros((3, n), np.float32)
    fl = np.zeros(n, np.uint8)
    check(lib().tacchi_init_lattice(nx, ny, nz, pad_side, pad_bottom, seed, int(bool(jitter)),
                                    u.ctypes.data_as(C.POINTER(C.c_float)),
                                    fl.ctypes.data_as(C.POINTER(C.c_uint8))), "tacchi_init_lattice")
    return u, fl


def shade(H, pixel_x, pixel_y, z_top, rp=None, out=None, stream=None):
    """Phong shading (Eqs. 12-14) of a device height map H [h, w] (metres)."""
    torch = _torch()
    rp = rp or default_render_params()
    h, w = H.shape
    H = H.contiguous().float()
    out = out if out is not None else torch.empty((h, w, 3), device=H.device, dtype=torch.float32)
    check(lib().tacchi_shade(C.byref(rp), ptr(H), w, h, pixel_x, pixel_y, z_top, ptr(out),
                             _stream_handle(torch, stream)), "tacchi_shade")
    return out


class Tacchi:
    """One simulated sensor elastomer (a tacchi_handle)."""

    def __init__(self, extent_m, dx, E=3.0e5, nu=0.45, density=1000.0, seed=0, jitter=True,
                 pad_side=4, pad_bottom=3, pad_top=4, gravity=(0.0, 0.0, 0.0), fix_base=True,
                 block=None, stream=None, contact_mode=0):
        torch = _torch()
        self._torch = torch
        d = _lib.ElastomerDesc()
        for a in range(3):
            d.extent_m[a] = extent_m[a]
            d.gravity[a] = gravity[a]
        d.dx_m, d.E_pa, d.nu, d.density = dx, E, nu, density
        d.seed, d.jitter = seed, int(bool(jitter))
        d.pad_side, d.pad_bottom, d.pad_top = pad_side, pad_bottom, pad_top
        d.free_base = 0 if fix_base else 1
        d.contact_mode = int(contact_mode)
        if block is not None:
            for a in range(3):
                d.block[a] = block[a]
            if len(block) > 3:
                d.threads_per_cell = block[3]
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        self._h = None
        check(lib().tacchi_create(C.byref(d), C.c_void_p(self._stream.cuda_stream), C.byref(h)),
              "tacchi_create")
        self._h = h
        info = _lib.Info()
        check(lib().tacchi_info(self._h, C.byref(info)), "tacchi_info")
        self.N = int(info.n_particles)
        self.n_surface = int(info.n_surface)
        self.grid = tuple(int(x) for x in info.grid)
        self.n_nodes = int(info.n_nodes)
        self.origin = tuple(float(x) for x in info.origin_m)
        self.dx = float(info.dx_m)
        self.z_top = float(info.z_top_m)
        self.block = tuple(int(x) for x in info.block)
        self.threads_per_cell = int(info.threads_per_cell)
        self.n_blocks = int(info.n_blocks)
        self.device_bytes = int(info.device_bytes)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.extent = tuple(float(x) for x in extent_m)

    def close(self):
        if getattr(self, "_h", None):
            lib().tacchi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- indenter ---------------------------------------------------------
    def set_indenter(self, kind=None, params=(), pose=None, vel=None, hm=None, hm_pixel=0.0):
        dp = None
        keep = None
        if kind is not None:
            dp = _lib.IndenterDesc()
            dp.kind = int(kind)
            for e, x in enumerate(params):
                dp.params[e] = x
            if hm is not None:
                keep = np.ascontiguousarray(hm, np.float32)
                dp.hm_h, dp.hm_w = keep.shape
                dp.hm_pixel_m = hm_pixel
                dp.hm = keep.ctypes.data_as(C.POINTER(C.c_float))
        pz = None if pose is None else (C.c_double * 7)(*pose)
        vz = None if vel is None else (C.c_double * 6)(*vel)
        check(lib().tacchi_set_indenter(self._h, C.byref(dp) if dp is not None else None, pz, vz),
              "tacchi_set_indenter")
        del keep

    def indenter_pose(self):
        p = (C.c_double * 7)()
        check(lib().tacchi_get_indenter_pose(self._h, p), "tacchi_get_indenter_pose")
        return tuple(p)

    # -- stepping -----------------------------------------------------------
    def step(self, n_substeps, dt):
        check(lib().tacchi_step(self._h, int(n_substeps), float(dt)), "tacchi_step")

    def sync(self):
        check(lib().tacchi_sync(self._h), "tacchi_sync")

    def status(self) -> int:
        """Synchronise and return the device status code (0 = OK)."""
        return int(lib().tacchi_sync(self._h))

    def set_transfer(self, shape, threads_per_cell):
        """Transfer plan: sort block (bx, by, bz) and threads sharing a cell (1 or 3)."""
        check(lib().tacchi_set_transfer(self._h, *shape, int(threads_per_cell)), "tacchi_set_transfer")
        self.block, self.threads_per_cell = tuple(int(x) for x in shape), int(threads_per_cell)

    def autotune(self, n_substeps, dt):
        """Times every transfer plan on the current state (restored after);
        keeps the fastest and returns ((bx, by, bz, threads per cell),
        {plan name: ms per substep})."""
        best = (C.c_int * 4)()
        ms = (C.c_double * len(TRANSFER_PLANS))()
        check(lib().tacchi_autotune(self._h, int(n_substeps), float(dt), best, ms), "tacchi_autotune")
        self.block, self.threads_per_cell = tuple(best[:3]), int(best[3])
        return tuple(best), dict(zip(TRANSFER_PLANS, list(ms)))

    def set_launch(self, persistent):
        """Step as one persistent cooperative kernel per chunk (True) or as a
        CUDA graph of kernels (False, the default)."""
        check(lib().tacchi_set_launch(self._h, 1 if persistent else 0), "tacchi_set_launch")

    def set_barrier_wait(self, max_polls, extra_arrivals=0):
        check(lib().tacchi_set_barrier_wait(self._h, int(max_polls), int(extra_arrivals)), "tacchi_set_barrier_wait")

    def set_pipeline(self, on):
        """Fused transfers by the pipelined kernel (True, the default where the
        plan has one) or by one CTA per sort block (False)."""
        check(lib().tacchi_set_pipeline(self._h, 1 if on else 0), "tacchi_set_pipeline")

    @property
    def pipelined(self):
        info = _lib.Info()
        check(lib().tacchi_info(self._h, C.byref(info)), "tacchi_info")
        return bool(info.pipelined)

    def set_profiling(self, on=True):
        check(lib().tacchi_set_profiling(self._h, int(bool(on))), "tacchi_set_profiling")

    def profile(self, reset=False):
        p = _lib.Profile()
        check(lib().tacchi_get_profile(self._h, C.byref(p), int(bool(reset))), "tacchi_get_profile")
        return {f: getattr(p, f) for f, _ in p._fields_}

    def clear_error(self):
        check(lib().tacchi_clear_error(self._h), "tacchi_clear_error")

    # -- rendering ------------------------------------------------------------
    def _window(self, window):
        if window is None:  # the whole top face
            window = (0.0, 0.0, self.extent[0], self.extent[1])
        return (C.c_double * 4)(*window)

    def heightmap(self, w, h, window=None, fill_radius=8, out=None):
        torch = self._torch
        out = out if out is not None else torch.empty((h, w), device=self.device, dtype=torch.float32)
        check(lib().tacchi_heightmap(self._h, w, h, self._window(window), fill_radius, ptr(out)),
              "tacchi_heightmap")
        return out

    def render(self, w, h, window=None, rp=None, fill_radius=8, out=None, out_height=None):
        torch = self._torch
        rp = rp or default_render_params()
        out = out if out is not None else torch.empty((h, w, 3), device=self.device, dtype=torch.float32)
        check(lib().tacchi_render(self._h, C.byref(rp), w, h, self._window(window), fill_radius,
                                  ptr(out), ptr(out_height)), "tacchi_render")
        return out

    def render_smoothed(self, w, h, sigma_m, window=None, rp=None, out=None, out_height=None):
        """Comparison renderer: the indenter's depth map smoothed by a
        Gaussian of standard deviation sigma_m, shaded (see TacchiBatch)."""
        torch = self._torch
        rp = rp or default_render_params()
        out = out if out is not None else torch.empty((h, w, 3), device=self.device, dtype=torch.float32)
        check(lib().tacchi_render_smoothed(self._h, C.byref(rp), w, h, self._window(window), float(sigma_m),
                                           ptr(out), ptr(out_height)), "tacchi_render_smoothed")
        return out

    # -- state ----------------------------------------------------------------
    def get_state(self):
        torch = self._torch
        n = self.N
        f = lambda *s: torch.empty(s, device=self.device, dtype=torch.float32)
        u, v, Cm, Fm = f(3, n), f(3, n), f(9, n), f(9, n)
        flags = torch.empty(n, device=self.device, dtype=torch.uint8)
        st = lib().tacchi_get_state(self._h, ptr(u), ptr(v), ptr(Cm), ptr(Fm), ptr(flags))
        return dict(u=u, v=v, C=Cm, Fm=Fm, flags=flags, status=int(st))

    def set_state(self, u, v=None, Cm=None, Fm=None):
        torch = self._torch
        dev = lambda t, r: None if t is None else torch.as_tensor(t, dtype=torch.float32).reshape(
            r, self.N).contiguous().to(self.device)
        tu, tv, tC, tF = dev(u, 3), dev(v, 3), dev(Cm, 9), dev(Fm, 9)
        check(lib().tacchi_set_state(self._h, ptr(tu), ptr(tv), ptr(tC), ptr(tF)), "tacchi_set_state")
        check(lib().tacchi_sync(self._h), "tacchi_set_state")

    def set_indenter_particles(self, pts, mass):
        """Indenter represented by particles (see TacchiBatch)."""
        a = np.ascontiguousarray(np.asarray(pts, np.float32).reshape(-1, 3))
        check(lib().tacchi_set_indenter_particles(self._h, a.shape[0], a.ctypes.data_as(C.POINTER(C.c_float)),
                                                  float(mass)), "tacchi_set_indenter_particles")

    def markers(self, xy, out=None):
        """Marker displacement (m) at rest positions xy [n, 2] (see
        TacchiBatch.markers)."""
        torch = self._torch
        xy = torch.as_tensor(xy, dtype=torch.float32, device=self.device).reshape(-1, 2).contiguous()
        out = out if out is not None else torch.empty((xy.shape[0], 3), device=self.device, dtype=torch.float32)
        check(lib().tacchi_batch_markers(self._h, 0, xy.shape[0], ptr(xy), ptr(out)), "tacchi_batch_markers")
        return out

    def get_grid(self):
        """[n_nodes, 4] = (M, MG) of the last particle-to-grid transfer."""
        torch = self._torch
        out = torch.empty((self.n_nodes, 4), device=self.device, dtype=torch.float32)
        check(lib().tacchi_get_grid(self._h, ptr(out)), "tacchi_get_grid")
        self.sync()
        return out


def _desc_from(block, seed=None, fix_base=True, gravity=(0.0, 0.0, 0.0), sort_block=None, jitter=True,
               contact_mode=0):
    """ElastomerDesc from an object with nx, ny, nz, dx, E, nu, rho, pad_side,
    pad_bottom, pad_top and seed attributes."""
    d = _lib.ElastomerDesc()
    ext = (block.nx * block.dx, block.ny * block.dx, block.nz * block.dx)
    for a in range(3):
        d.extent_m[a] = ext[a]
        d.gravity[a] = gravity[a]
    d.dx_m, d.E_pa, d.nu, d.density = block.dx, block.E, block.nu, block.rho
    d.seed = block.seed if seed is None else seed
    d.jitter = int(bool(jitter))
    d.pad_side, d.pad_bottom, d.pad_top = block.pad_side, block.pad_bottom, block.pad_top
    d.free_base = 0 if fix_base else 1
    d.contact_mode = int(contact_mode)
    if sort_block is not None:
        for a in range(3):
            d.block[a] = sort_block[a]
        if len(sort_block) > 3:
            d.threads_per_cell = sort_block[3]
    return d


class TacchiBatch:
    """Many independent sensor elastomers advanced together (one handle)."""

    def __init__(self, blocks, fix_base=True, sort_block=None, stream=None, contact_mode=0):
        torch = _torch()
        self._torch = torch
        n = len(blocks)
        arr = (_lib.ElastomerDesc * n)()
        for i, b in enumerate(blocks):
            arr[i] = _desc_from(b, fix_base=fix_base, sort_block=sort_block, contact_mode=contact_mode)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        self._h = None
        check(lib().tacchi_batch_create(n, arr, C.c_void_p(self._stream.cuda_stream), C.byref(h)),
              "tacchi_batch_create")
        self._h = h
        self.n = n
        self.blocks = list(blocks)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.info = []
        for i in range(n):
            info = _lib.Info()
            check(lib().tacchi_batch_info(self._h, i, C.byref(info)), "tacchi_batch_info")
            self.info.append(dict(N=int(info.n_particles), n_surface=int(info.n_surface),
                                  grid=tuple(info.grid), n_nodes=int(info.n_nodes),
                                  origin=tuple(info.origin_m), dx=float(info.dx_m),
                                  z_top=float(info.z_top_m)))
        self.N_total = sum(x["N"] for x in self.info)

    def close(self):
        if getattr(self, "_h", None):
            lib().tacchi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_indenter(self, i, kind=None, params=(), pose=None, vel=None, hm=None, hm_pixel=0.0):
        dp = None
        keep = None
        if kind is not None:
            dp = _lib.IndenterDesc()
            dp.kind = int(kind)
            for e, x in enumerate(params):
                dp.params[e] = x
            if hm is not None:
                keep = np.ascontiguousarray(hm, np.float32)
                dp.hm_h, dp.hm_w = keep.shape
                dp.hm_pixel_m = hm_pixel
                dp.hm = keep.ctypes.data_as(C.POINTER(C.c_float))
        pz = None if pose is None else (C.c_double * 7)(*pose)
        vz = None if vel is None else (C.c_double * 6)(*vel)
        check(lib().tacchi_batch_set_indenter(self._h, i, C.byref(dp) if dp is not None else None,
                                              pz, vz), "tacchi_batch_set_indenter")
        del keep

    def indenter_pose(self, i):
        p = (C.c_double * 7)()
        check(lib().tacchi_batch_get_indenter_pose(self._h, i, p), "tacchi_batch_get_indenter_pose")
        return tuple(p)

    def step(self, n_substeps, dt):
        check(lib().tacchi_step(self._h, int(n_substeps), float(dt)), "tacchi_step")

    def sync(self):
        check(lib().tacchi_sync(self._h), "tacchi_sync")

    def status(self) -> int:
        return int(lib().tacchi_sync(self._h))

    def set_profiling(self, on=True):
        check(lib().tacchi_set_profiling(self._h, int(bool(on))), "tacchi_set_profiling")

    def profile(self, reset=False):
        p = _lib.Profile()
        check(lib().tacchi_get_profile(self._h, C.byref(p), int(bool(reset))), "tacchi_get_profile")
        return {f: getattr(p, f) for f, _ in p._fields_}

    def reset(self):
        """Every instance back to its initial lattice (indenters kept)."""
        check(lib().tacchi_batch_reset(self._h), "tacchi_batch_reset")

    def set_block(self, shape):
        """Sort block (bx, by, bz) with one thread per cell."""
        check(lib().tacchi_set_block(self._h, *shape), "tacchi_set_block")

    def set_transfer(self, shape, threads_per_cell):
        """Transfer plan: sort block (bx, by, bz) and threads sharing a cell (1 or 3)."""
        check(lib().tacchi_set_transfer(self._h, *shape, int(threads_per_cell)), "tacchi_set_transfer")

    def set_launch(self, persistent):
        """Step as one persistent cooperative kernel per chunk (True) or as a
        CUDA graph of kernels (False, the default)."""
        check(lib().tacchi_set_launch(self._h, 1 if persistent else 0), "tacchi_set_launch")

    def set_barrier_wait(self, max_polls, extra_arrivals=0):
        check(lib().tacchi_set_barrier_wait(self._h, int(max_polls), int(extra_arrivals)), "tacchi_set_barrier_wait")

    def set_pipeline(self, on):
        """Fused transfers by the pipelined kernel (True, the default where the
        plan has one) or by one CTA per sort block (False)."""
        check(lib().tacchi_set_pipeline(self._h, 1 if on else 0), "tacchi_set_pipeline")

    @property
    def pipelined(self):
        info = _lib.Info()
        check(lib().tacchi_info(self._h, C.byref(info)), "tacchi_info")
        return bool(info.pipelined)

    def transfer_plan(self):
        info = _lib.Info()
        check(lib().tacchi_info(self._h, C.byref(info)), "tacchi_info")
        return tuple(int(x) for x in info.block), int(info.threads_per_cell)

    def autotune(self, n_substeps, dt):
        """Times every transfer plan; returns ((bx, by, bz, threads per
        cell) of the fastest, {plan name: ms per substep})."""
        best = (C.c_int * 4)()
        ms = (C.c_double * len(TRANSFER_PLANS))()
        check(lib().tacchi_autotune(self._h, int(n_substeps), float(dt), best, ms), "tacchi_autotune")
        return tuple(best), dict(zip(TRANSFER_PLANS, list(ms)))

    def heightmap(self, i, w, h, window, fill_radius=8, out=None):
        torch = self._torch
        out = out if out is not None else torch.empty((h, w), device=self.device, dtype=torch.float32)
        check(lib().tacchi_batch_heightmap(self._h, i, w, h, (C.c_double * 4)(*window), fill_radius,
                                           ptr(out)), "tacchi_batch_heightmap")
        return out

    def render(self, i, w, h, window, rp=None, fill_radius=8, out=None, out_height=None):
        torch = self._torch
        rp = rp or default_render_params()
        out = out if out is not None else torch.empty((h, w, 3), device=self.device, dtype=torch.float32)
        check(lib().tacchi_batch_render(self._h, i, C.byref(rp), w, h, (C.c_double * 4)(*window),
                                        fill_radius, ptr(out), ptr(out_height)), "tacchi_batch_render")
        return out

    def render_smoothed(self, i, w, h, window, sigma_m, rp=None, out=None, out_height=None):
        """The depth-smoothing renderers of Sec. II, for comparison: the
        indenter's penetration map convolved with a Gaussian of standard
        deviation sigma_m (m, truncated at 3 sigma), H = z_top - that, shaded
        by Eqs. 12-14.  No physics."""
        torch = self._torch
        rp = rp or default_render_params()
        out = out if out is not None else torch.empty((h, w, 3), device=self.device, dtype=torch.float32)
        check(lib().tacchi_batch_render_smoothed(self._h, i, C.byref(rp), w, h, (C.c_double * 4)(*window),
                                                 float(sigma_m), ptr(out), ptr(out_height)),
              "tacchi_batch_render_smoothed")
        return out

    def displacement_map(self, i, w, h, window, out=None):
        torch = self._torch
        out = out if out is not None else torch.empty((h, w, 3), device=self.device, dtype=torch.float32)
        check(lib().tacchi_batch_displacement_map(self._h, i, w, h, (C.c_double * 4)(*window), ptr(out)),
              "tacchi_batch_displacement_map")
        return out

    def set_indenter_particles(self, i, pts, mass):
        """Represent instance i's indenter by particles at local positions
        pts (m, [n, 3]) of the given mass each (the paper's Eq. 10 model); an
        empty array returns it to the grid-boundary indenter."""
        a = np.ascontiguousarray(np.asarray(pts, np.float32).reshape(-1, 3))
        check(lib().tacchi_batch_set_indenter_particles(self._h, i, a.shape[0], a.ctypes.data_as(C.POINTER(C.c_float)),
                                                        float(mass)), "tacchi_batch_set_indenter_particles")

    def markers(self, i, xy, out=None):
        """Displacement (m) of the markers at rest positions xy [n, 2] (m,
        world, on the top face): each follows the top-layer particle whose
        rest sub-cell contains it."""
        torch = self._torch
        xy = torch.as_tensor(xy, dtype=torch.float32, device=self.device).reshape(-1, 2).contiguous()
        n = xy.shape[0]
        out = out if out is not None else torch.empty((n, 3), device=self.device, dtype=torch.float32)
        check(lib().tacchi_batch_markers(self._h, i, n, ptr(xy), ptr(out)), "tacchi_batch_markers")
        return out

    def penetration_map(self, i, w, h, window, out=None):
        torch = self._torch
        out = out if out is not None else torch.empty((h, w), device=self.device, dtype=torch.float32)
        check(lib().tacchi_batch_penetration_map(self._h, i, w, h, (C.c_double * 4)(*window), ptr(out)),
              "tacchi_batch_penetration_map")
        return out

    def get_state(self, i):
        torch = self._torch
        n = self.info[i]["N"]
        f = lambda *s: torch.empty(s, device=self.device, dtype=torch.float32)
        u, v, Cm, Fm = f(3, n), f(3, n), f(9, n), f(9, n)
        flags = torch.empty(n, device=self.device, dtype=torch.uint8)
        st = lib().tacchi_batch_get_state(self._h, i, ptr(u), ptr(v), ptr(Cm), ptr(Fm), ptr(flags))
        return dict(u=u, v=v, C=Cm, Fm=Fm, flags=flags, status=int(st))

    def set_state(self, i, u, v=None, Cm=None, Fm=None):
        torch = self._torch
        n = self.info[i]["N"]
        dev = lambda t, r: None if t is None else torch.as_tensor(t, dtype=torch.float32).reshape(
            r, n).contiguous().to(self.device)
        tu, tv, tC, tF = dev(u, 3), dev(v, 3), dev(Cm, 9), dev(Fm, 9)
        check(lib().tacchi_batch_set_state(self._h, i, ptr(tu), ptr(tv), ptr(tC), ptr(tF)),
              "tacchi_batch_set_state")
        check(lib().tacchi_sync(self._h), "tacchi_batch_set_state")


class SurrogateNet:
    """The learned surrogate (a tacchi_nn handle): U-Net trained and run by
    the library's BF16 tensor-core kernels; inputs/outputs are FP32 NHWC
    device tensors."""

    def __init__(self, widths=(32, 64, 128, 256), in_channels=2, out_channels=3, size=64,
                 max_batch=256, seed=0, stream=None):
        torch = _torch()
        self._torch = torch
        self.widths = tuple(widths)
        self.cin, self.cout, self.size, self.max_batch = in_channels, out_channels, size, max_batch
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        w = (C.c_int * len(widths))(*widths)
        h = C.c_void_p()
        self._h = None
        check(lib().tacchi_nn_create(len(widths), w, in_channels, out_channels, size, size, max_batch,
                                     seed, C.c_void_p(self._stream.cuda_stream), C.byref(h)),
              "tacchi_nn_create")
        self._h = h
        n = C.c_int64()
        check(lib().tacchi_nn_num_params(self._h, C.byref(n)), "tacchi_nn_num_params")
        self.num_params = int(n.value)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None):
            lib().tacchi_nn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self, grads=False):
        out = np.zeros(self.num_params, np.float32)
        check(lib().tacchi_nn_get_params(self._h, int(bool(grads)), out.ctypes.data_as(C.POINTER(C.c_float))),
              "tacchi_nn_get_params")
        return out

    def set_params(self, vec):
        v = np.ascontiguousarray(vec, np.float32)
        assert v.size == self.num_params
        check(lib().tacchi_nn_set_params(self._h, v.ctypes.data_as(C.POINTER(C.c_float))), "tacchi_nn_set_params")

    def _dev(self, t):
        return self._torch.as_tensor(t, dtype=self._torch.float32, device=self.device).contiguous()

    def forward(self, x, out=None):
        x = self._dev(x)
        b = x.shape[0]
        out = out if out is not None else self._torch.empty((b, self.size, self.size, self.cout), device=self.device)
        check(lib().tacchi_nn_forward(self._h, b, ptr(x), ptr(out)), "tacchi_nn_forward")
        return out

    def gradients(self, x, target):
        x, t = self._dev(x), self._dev(target)
        loss = C.c_float()
        check(lib().tacchi_nn_gradients(self._h, x.shape[0], ptr(x), ptr(t), C.byref(loss)), "tacchi_nn_gradients")
        return float(loss.value)

    def train_step(self, x, target, lr, want_loss=True):
        x, t = self._dev(x), self._dev(target)
        loss = C.c_float()
        check(lib().tacchi_nn_train_step(self._h, x.shape[0], ptr(x), ptr(t), float(lr),
                                         C.byref(loss) if want_loss else None), "tacchi_nn_train_step")
        return float(loss.value) if want_loss else None
