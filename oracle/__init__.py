"""FP64 CPU oracle of the Tacchi method (arXiv 2301.08343, Sec. III).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product package never imports
it.  The C source (``tacchi_oracle.c``) is compiled here with gcc into
``liboracle.so``; this module only marshals numpy arrays through ctypes.

Parity status per function (pins live in ``tests/test_oracle_*.py``):
  weights, P2G (Eqs. 2-5), grid update (Eq. 6 + boundaries), G2P and
  advection (Eqs. 7-11), polar/stress, lattice, height map, shading
  (Eqs. 12-14): pinned.  Absolute image colours depend on light constants the
  paper delegates to another work, so only their self-consistency is pinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tacchi_oracle.c")
_HDR = os.path.join(_HERE, "tacchi_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

IND_NONE, IND_SPHERE, IND_CYLINDER, IND_CONE, IND_PRISM, IND_HEIGHTMAP = range(6)
ERR_OUT_OF_GRID = 1
ERR_NUMERICAL = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, OpenMP, no FP contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("pad_side", C.c_int), ("pad_bottom", C.c_int), ("pad_top", C.c_int),
                ("dx", C.c_double), ("E", C.c_double), ("nu", C.c_double),
                ("rho", C.c_double), ("gravity", C.c_double * 3), ("fix_base", C.c_int),
                ("slip", C.c_int)]


class RenderParams(C.Structure):
    _fields_ = [("n_lights", C.c_int), ("dir", (C.c_double * 3) * 8),
                ("diffuse", (C.c_double * 3) * 8), ("specular", (C.c_double * 3) * 8),
                ("ambient", C.c_double * 3), ("ka", C.c_double), ("kd", C.c_double),
                ("ks", C.c_double), ("alpha", C.c_double)]


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            dp, fp, u8p, ip = (C.POINTER(C.c_double), C.POINTER(C.c_float),
                               C.POINTER(C.c_uint8), C.POINTER(C.c_int))
            L.ora_lattice.argtypes = [C.c_int] * 5 + [C.c_uint64, C.c_int, fp, u8p]
            L.ora_splitmix64_at.argtypes = [C.c_uint64, C.c_uint64]
            L.ora_splitmix64_at.restype = C.c_uint64
            L.ora_create.argtypes = [C.POINTER(Params)]
            L.ora_create.restype = C.c_void_p
            L.ora_destroy.argtypes = [C.c_void_p]
            L.ora_num_particles.argtypes = [C.c_void_p]
            L.ora_num_particles.restype = C.c_longlong
            L.ora_grid_dims.argtypes = [C.c_void_p, ip]
            L.ora_set_threads.argtypes = [C.c_int]
            L.ora_set_state.argtypes = [C.c_void_p, fp, fp, fp, fp, u8p]
            L.ora_set_rest.argtypes = [C.c_void_p, fp]
            L.ora_get_state.argtypes = [C.c_void_p, dp, dp, dp, dp]
            L.ora_get_state_f32.argtypes = [C.c_void_p, fp, fp, fp, fp]
            L.ora_set_indenter.argtypes = [C.c_void_p, C.c_int, dp, C.c_int, C.c_int,
                                           C.c_double, fp, dp, dp]
            L.ora_get_pose.argtypes = [C.c_void_p, dp]
            L.ora_set_indenter_particles.argtypes = [C.c_void_p, C.c_longlong, dp, C.c_double]
            L.ora_node_inside.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
            L.ora_p2g.argtypes = [C.c_void_p, C.c_double, dp, dp]
            L.ora_substep.argtypes = [C.c_void_p, C.c_double]
            L.ora_run.argtypes = [C.c_void_p, C.c_int, C.c_double]
            L.ora_g2p.argtypes = [C.c_void_p, dp, C.c_double]
            L.ora_last_grid.argtypes = [C.c_void_p, dp, dp]
            L.ora_last_grid_velocity.argtypes = [C.c_void_p, dp]
            L.ora_weights.argtypes = [dp, ip, dp]
            L.ora_polar.argtypes = [dp, dp]
            L.ora_stress.argtypes = [dp, C.c_double, C.c_double, dp]
            L.ora_heightmap.argtypes = [C.c_void_p, dp, C.c_int, C.c_int, C.c_int, dp]
            L.ora_shade.argtypes = [dp, C.c_int, C.c_int, C.c_double, C.c_double,
                                    C.c_double, C.POINTER(RenderParams), dp]
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().ora_set_threads(int(n))


def splitmix64_at(seed: int, counter: int) -> int:
    return int(lib().ora_splitmix64_at(seed, counter))


def lattice(nx, ny, nz, pad_side, pad_bottom, seed, jitter=True):
    """Initial particle positions (cells, FP32, [3][N]) and flags (uint8)."""
    n = 8 * nx * ny * nz
    u = np.zeros((3, n), np.float32)
    fl = np.zeros(n, np.uint8)
    lib().ora_lattice(nx, ny, nz, pad_side, pad_bottom, seed, int(bool(jitter)),
                      _p(u, C.c_float), _p(fl, C.c_uint8))
    return u, fl


def weights(xi):
    xi = np.ascontiguousarray(xi, np.float64)
    base = np.zeros(3, np.int32)
    w = np.zeros(27, np.float64)
    lib().ora_weights(_p(xi, C.c_double), _p(base, C.c_int), _p(w, C.c_double))
    return base, w.reshape(3, 3, 3)  # [k][j][i]


def polar(F):
    F = np.ascontiguousarray(F, np.float64).reshape(9)
    R = np.zeros(9)
    lib().ora_polar(_p(F, C.c_double), _p(R, C.c_double))
    return R.reshape(3, 3)


def stress(F, mu, la):
    F = np.ascontiguousarray(F, np.float64).reshape(9)
    t = np.zeros(9)
    lib().ora_stress(_p(F, C.c_double), mu, la, _p(t, C.c_double))
    return t.reshape(3, 3)


def shade(H, pixel_x, pixel_y, z_top, rp: RenderParams):
    H = np.ascontiguousarray(H, np.float64)
    h, w = H.shape
    out = np.zeros((h, w, 3))
    lib().ora_shade(_p(H, C.c_double), w, h, pixel_x, pixel_y, z_top, C.byref(rp),
                    _p(out, C.c_double))
    return out


def render_params(n_lights, dirs, diffuse, specular, ambient, ka, kd, ks, alpha):
    rp = RenderParams()
    rp.n_lights = n_lights
    for m in range(n_lights):
        for a in range(3):
            rp.dir[m][a] = dirs[m][a]
            rp.diffuse[m][a] = diffuse[m][a]
            rp.specular[m][a] = specular[m][a]
    for a in range(3):
        rp.ambient[a] = ambient[a]
    rp.ka, rp.kd, rp.ks, rp.alpha = ka, kd, ks, alpha
    return rp


class Sim:
    """One elastomer instance simulated by the oracle (FP64)."""

    def __init__(self, nx, ny, nz, dx, E, nu, rho, pad_side=4, pad_bottom=3, pad_top=4,
                 gravity=(0.0, 0.0, 0.0), fix_base=True, slip=False):
        p = Params()
        p.nx, p.ny, p.nz = nx, ny, nz
        p.pad_side, p.pad_bottom, p.pad_top = pad_side, pad_bottom, pad_top
        p.dx, p.E, p.nu, p.rho = dx, E, nu, rho
        for a in range(3):
            p.gravity[a] = gravity[a]
        p.fix_base = int(bool(fix_base))
        p.slip = int(bool(slip))
        self.params = p
        self._L = lib()
        self._h = self._L.ora_create(C.byref(p))
        self.N = int(self._L.ora_num_particles(self._h))
        d = np.zeros(3, np.int32)
        self._L.ora_grid_dims(self._h, _p(d, C.c_int))
        self.G = tuple(int(x) for x in d)  # nodes per axis (x, y, z)
        self.nodes = int(np.prod(self.G))
        self.dx = dx
        self.origin = np.array([-pad_side * dx, -pad_side * dx, -pad_bottom * dx])
        self.z_top = nz * dx
        self.V0 = dx ** 3 / 8.0
        self.m = rho * self.V0
        self.mu = E / (2 * (1 + nu))
        self.la = E * nu / ((1 + nu) * (1 - 2 * nu))

    def __del__(self):
        try:
            if self._h:
                self._L.ora_destroy(self._h)
                self._h = None
        except Exception:
            pass

    def set_state(self, u, v=None, Cm=None, Fm=None, flags=None):
        f32 = lambda a: None if a is None else np.ascontiguousarray(a, np.float32)
        u, v, Cm, Fm = f32(u), f32(v), f32(Cm), f32(Fm)
        fl = None if flags is None else np.ascontiguousarray(flags, np.uint8)
        self._L.ora_set_state(self._h, _p(u, C.c_float), _p(v, C.c_float),
                              _p(Cm, C.c_float), _p(Fm, C.c_float), _p(fl, C.c_uint8))

    def set_rest(self, u0):
        u0 = np.ascontiguousarray(u0, np.float32)
        self._L.ora_set_rest(self._h, _p(u0, C.c_float))

    def state(self):
        n = self.N
        xi, v, Cm, F = (np.zeros((3, n)), np.zeros((3, n)), np.zeros((9, n)), np.zeros((9, n)))
        self._L.ora_get_state(self._h, _p(xi, C.c_double), _p(v, C.c_double),
                              _p(Cm, C.c_double), _p(F, C.c_double))
        return xi, v, Cm, F

    def state_f32(self):
        n = self.N
        u, v, Cm, Fm = (np.zeros((3, n), np.float32), np.zeros((3, n), np.float32),
                        np.zeros((9, n), np.float32), np.zeros((9, n), np.float32))
        self._L.ora_get_state_f32(self._h, _p(u, C.c_float), _p(v, C.c_float),
                                  _p(Cm, C.c_float), _p(Fm, C.c_float))
        return u, v, Cm, Fm

    def set_indenter(self, kind, params=(), pose=(0, 0, 0, 1, 0, 0, 0), vel=(0,) * 6,
                     hm=None, hm_pixel=0.0):
        pr = np.zeros(8)
        pr[:len(params)] = params
        pose = np.ascontiguousarray(pose, np.float64)
        vel = np.ascontiguousarray(vel, np.float64)
        hmw = hmh = 0
        hma = None
        if hm is not None:
            hma = np.ascontiguousarray(hm, np.float32)
            hmh, hmw = hma.shape
        rc = self._L.ora_set_indenter(self._h, kind, _p(pr, C.c_double), hmw, hmh,
                                      float(hm_pixel), _p(hma, C.c_float),
                                      _p(pose, C.c_double), _p(vel, C.c_double))
        if rc != 0:
            raise ValueError("oracle rejected the indenter description")

    def set_indenter_particles(self, pts, mass):
        """Indenter represented by particles at local positions pts (m,
        [n, 3]), each of the given mass (Eq. 10, p in I); an empty array
        restores the grid-boundary indenter."""
        a = np.ascontiguousarray(np.asarray(pts, np.float64).reshape(-1, 3))
        rc = self._L.ora_set_indenter_particles(self._h, a.shape[0], _p(a, C.c_double), float(mass))
        if rc != 0:
            raise ValueError("oracle rejected the indenter particles")

    def pose(self):
        p = np.zeros(7)
        self._L.ora_get_pose(self._h, _p(p, C.c_double))
        return p

    def node_inside(self, i, j, k) -> bool:
        return bool(self._L.ora_node_inside(self._h, i, j, k))

    def p2g(self, dt):
        m = np.zeros(self.nodes)
        mom = np.zeros((3, self.nodes))
        self._L.ora_p2g(self._h, dt, _p(m, C.c_double), _p(mom, C.c_double))
        return m, mom

    def substep(self, dt) -> int:
        return int(self._L.ora_substep(self._h, dt))

    def run(self, n, dt) -> int:
        return int(self._L.ora_run(self._h, n, dt))

    def g2p(self, V, dt) -> int:
        """Eqs. 7-11 alone from the grid velocity V ([3][nodes], m/s)."""
        V = np.ascontiguousarray(V, np.float64).reshape(3, self.nodes)
        return int(self._L.ora_g2p(self._h, _p(V, C.c_double), dt))

    def last_grid(self):
        m = np.zeros(self.nodes)
        mom = np.zeros((3, self.nodes))
        self._L.ora_last_grid(self._h, _p(m, C.c_double), _p(mom, C.c_double))
        return m, mom

    def last_grid_velocity(self):
        V = np.zeros((3, self.nodes))
        self._L.ora_last_grid_velocity(self._h, _p(V, C.c_double))
        return V

    def heightmap(self, window, w, h, fill_radius=8):
        win = np.ascontiguousarray(window, np.float64)
        H = np.zeros((h, w))
        self._L.ora_heightmap(self._h, _p(win, C.c_double), w, h, fill_radius,
                              _p(H, C.c_double))
        return H

    def node_positions(self):
        """World positions of all grid nodes, [3][nodes] (x fastest)."""
        gx, gy, gz = self.G
        k, j, i = np.meshgrid(np.arange(gz), np.arange(gy), np.arange(gx), indexing="ij")
        idx = np.stack([i.ravel(), j.ravel(), k.ravel()]).astype(np.float64)
        return self.origin[:, None] + idx * self.dx
