"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds no arithmetic of the method itself: only workload sizes,
random perturbations of particle states and procedural indenter height maps.
Both the CUDA path and the oracle are fed from here; neither is imported.

Workloads (sizes follow the paper's setup, Sec. IV-B, scaled as stated):
  C0  12 x 12 x 3 mm block, dX = 0.5 mm (24 x 24 x 6 cells), 8 particles per
      cell (27,648), E = 0.3 MPa, nu = 0.45, rho = 1000 kg/m^3, fixed base,
      sphere R = 3 mm pressing 1 mm over 500 substeps of dt = 1e-5 s,
      120 x 120 height map and image over the 12 x 12 mm top face.
  C1  32 x 24 x 4 mm block (GelSight-sized), dX = 0.1 mm (320 x 240 x 40
      cells, 24,576,000 particles), same material, dt = 1e-6 s, 640 x 480
      image; nine procedural indenters at depths 0.2-1.5 mm.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Block:
    nx: int
    ny: int
    nz: int
    dx: float
    E: float = 3.0e5
    nu: float = 0.45
    rho: float = 1000.0
    pad_side: int = 4
    pad_bottom: int = 3
    pad_top: int = 4
    seed: int = 0

    @property
    def n_particles(self) -> int:
        return 8 * self.nx * self.ny * self.nz

    @property
    def extent_m(self):
        return (self.nx * self.dx, self.ny * self.dx, self.nz * self.dx)


C0 = Block(24, 24, 6, 0.5e-3)
C0_DT = 1.0e-5
C0_SUBSTEPS = 500
C0_SPHERE_R = 3.0e-3
C0_SPEED = 1.0e-3 / (C0_SUBSTEPS * C0_DT)  # 1 mm over 500 substeps = 0.2 m/s
C0_IMAGE = (120, 120)

# 2 mm of grid above the gel and 1 mm at its sides leave room for the bulge
# a deep press of a large flat-backed indenter raises in the incompressible gel
C1 = Block(320, 240, 40, 0.1e-3, pad_side=10, pad_top=20)
C1_DT = 1.0e-6
C1_IMAGE = (640, 480)


def c0_sphere_pose():
    """Sphere centre over the block centre, tangent to the top face."""
    b = C0
    return (b.nx * b.dx / 2, b.ny * b.dx / 2, b.nz * b.dx + C0_SPHERE_R, 1.0, 0.0, 0.0, 0.0)


def c0_sphere_vel():
    return (0.0, 0.0, -C0_SPEED, 0.0, 0.0, 0.0)


def top_window(b: Block):
    """Window covering the whole top face, metres (x0, y0, x1, y1)."""
    return (0.0, 0.0, b.nx * b.dx, b.ny * b.dx)


def perturbed_state(u_rest: np.ndarray, seed: int, disp_cells=0.05, v_scale=0.05,
                    C_scale=20.0, F_scale=0.02):
    """A random particle state near rest: (u, v, C, Fm) in the shared FP32
    format (positions in cells, v in m/s, C in 1/s, Fm = F - I)."""
    rng = np.random.default_rng(seed)
    n = u_rest.shape[1]
    u = (u_rest + rng.uniform(-disp_cells, disp_cells, (3, n))).astype(np.float32)
    v = rng.normal(0.0, v_scale, (3, n)).astype(np.float32)
    Cm = rng.normal(0.0, C_scale, (9, n)).astype(np.float32)
    Fm = rng.normal(0.0, F_scale, (9, n)).astype(np.float32)
    return u, v, Cm, Fm


def random_rotations(n: int, seed: int) -> np.ndarray:
    """n random rotation matrices [n,3,3] from normalised Gaussian quaternions."""
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z); R[:, 0, 1] = 2 * (x * y - w * z); R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z); R[:, 1, 1] = 1 - 2 * (x * x + z * z); R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y); R[:, 2, 1] = 2 * (y * z + w * x); R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def default_lights():
    """Three RGB lights 120 degrees apart in azimuth, 30 degrees above the
    surface plane on the camera side; Phong constants of Eq. 12.  These are
    this project's defaults, not the calibrated GelSight constants."""
    dirs, dif, spe = [], [], []
    el = math.radians(30.0)
    cols = [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)]
    for m in range(3):
        az = math.radians(90.0 + 120.0 * m)
        dirs.append((math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), -math.sin(el)))
        dif.append(cols[m])
        spe.append((1.0, 1.0, 1.0))
    return dict(n_lights=3, dirs=dirs, diffuse=dif, specular=spe,
                ambient=(1.0, 1.0, 1.0), ka=0.2, kd=0.6, ks=0.2, alpha=5.0)


# --------------------------------------------------------------------------
# Procedural indenter height maps (protrusion heights in metres, >= 0).
def _grid(n, pix):
    c = (np.arange(n) + 0.5 - n / 2) * pix
    return np.meshgrid(c, c, indexing="xy")


def hm_dots(n=128, pix=0.1e-3, dot_r=0.25e-3, pitch=1.5e-3, count=5, height=1.0e-3):
    X, Y = _grid(n, pix)
    h = np.zeros_like(X)
    off = (np.arange(count) - (count - 1) / 2) * pitch
    for ox in off:
        for oy in off:
            h[(X - ox) ** 2 + (Y - oy) ** 2 <= dot_r ** 2] = height
    return h.astype(np.float32)


def hm_line(n=128, pix=0.1e-3, width=0.5e-3, length=10e-3, height=1.0e-3):
    X, Y = _grid(n, pix)
    h = np.where((np.abs(X) <= width / 2) & (np.abs(Y) <= length / 2), height, 0.0)
    return h.astype(np.float32)


def hm_wave(n=128, pix=0.1e-3, wavelength=2e-3, amp=0.5e-3):
    X, _ = _grid(n, pix)
    return (amp * (1.0 + np.cos(2 * np.pi * X / wavelength))).astype(np.float32)


def hm_perlin(n=128, pix=0.1e-3, seed=1, octaves=3, amp=1.0e-3):
    """Gradient-noise texture (sum of octaves of bilinearly blended random
    gradients with a quintic fade), rescaled to [0, amp]."""
    rng = np.random.default_rng(seed)
    acc = np.zeros((n, n))
    for o in range(octaves):
        cells = 4 * 2 ** o
        ang = rng.uniform(0, 2 * np.pi, (cells + 1, cells + 1))
        gx, gy = np.cos(ang), np.sin(ang)
        t = (np.arange(n) + 0.5) / n * cells
        i0 = np.minimum(t.astype(int), cells - 1)
        f = t - i0
        fy, fx = np.meshgrid(f, f, indexing="ij")
        iy, ix = np.meshgrid(i0, i0, indexing="ij")
        def dot(dx_, dy_):
            return gx[iy + dy_, ix + dx_] * (fx - dx_) + gy[iy + dy_, ix + dx_] * (fy - dy_)
        fade = lambda s: s * s * s * (s * (s * 6 - 15) + 10)
        ux, uy = fade(fx), fade(fy)
        n00, n10, n01, n11 = dot(0, 0), dot(1, 0), dot(0, 1), dot(1, 1)
        v = (n00 * (1 - ux) + n10 * ux) * (1 - uy) + (n01 * (1 - ux) + n11 * ux) * uy
        acc += v / 2 ** o
    acc -= acc.min()
    acc /= max(acc.max(), 1e-30)
    return (amp * acc).astype(np.float32)


def hm_worn_sphere(n=128, pix=0.1e-3, R=4e-3, cap=1.2e-3, seed=2, n_pits=60, pit_r=0.3e-3,
                   pit_d=0.15e-3):
    """A paraboloid cap (curvature radius R, height cap) with Poisson-placed
    pits: a worn spherical indenter."""
    X, Y = _grid(n, pix)
    rng = np.random.default_rng(seed)
    h = np.maximum(cap - (X ** 2 + Y ** 2) / (2 * R), 0.0)
    for _ in range(rng.poisson(n_pits)):
        cx, cy = rng.uniform(-n * pix / 2, n * pix / 2, 2)
        d2 = (X - cx) ** 2 + (Y - cy) ** 2
        h = np.where(d2 < pit_r ** 2, np.maximum(h - pit_d * (1 - d2 / pit_r ** 2), 0.0), h)
    return h.astype(np.float32)


# The nine procedural indenters of the GelSight-scale workload, each as
# (kind name, shape parameters, height map or None, tip offset above the
# pose's z): sphere R 4 mm, cylinder R 2 mm (lying, 10 mm long), cone of
# 60 degree apex angle, triangular prism (90 degree edge, 8 mm long), 5 x 5
# dot grid, 0.5 x 10 mm line, wave of 2 mm wavelength, gradient-noise texture
# and a pitted spherical cap.
C1_DEPTHS = (0.2e-3, 0.5e-3, 1.0e-3, 1.5e-3)


def c1_indenters():
    pix = 0.1e-3
    maps = {
        "dots": hm_dots(n=96, pix=pix),
        "line": hm_line(n=128, pix=pix),
        "wave": hm_wave(n=96, pix=pix),
        "perlin": hm_perlin(n=128, pix=pix, seed=1, octaves=3),
        "worn": hm_worn_sphere(n=96, pix=pix, seed=2),
    }
    out = [("sphere", (4e-3,), None, 4e-3),
           ("cylinder", (2e-3, 5e-3), None, 2e-3),
           ("cone", (math.radians(30.0), 5e-3), None, 0.0),
           ("prism", (math.radians(45.0), 4e-3, 3e-3), None, 0.0)]
    for name in ("dots", "line", "wave", "perlin", "worn"):
        hm = maps[name]
        out.append(("heightmap:" + name, (2e-3,), hm, float(hm.max())))
    return out


# --------------------------------------------------------------------------
# Batched workload: independent sensors of uneven sizes (C2).
C2_DX = 0.25e-3
C2_DT = 2.0e-6  # CFL about 0.27 at dx = 0.25 mm (P-wave speed 33.7 m/s)


def c2_instances(n=256, seed_base=1000):
    """n sensors: sides U[8, 16] mm, thickness U[2, 4] mm at dx = 0.25 mm,
    8 particles per cell; per instance an analytic indenter (sphere,
    cylinder, cone or prism) with random size, yaw U[0, pi), xy offset
    U[-1, 1] mm and depth U[0.1, 1.0] mm, all from numpy's PCG64 seeded with
    seed_base + i.  Returns [(Block, indenter dict)]."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed_base + i)
        nx = int(round(rng.uniform(8e-3, 16e-3) / C2_DX))
        ny = int(round(rng.uniform(8e-3, 16e-3) / C2_DX))
        nz = int(round(rng.uniform(2e-3, 4e-3) / C2_DX))
        blk = Block(nx, ny, nz, C2_DX, pad_side=6, pad_top=8, seed=seed_base + i)
        kind = ["sphere", "cylinder", "cone", "prism"][int(rng.integers(4))]
        yaw = rng.uniform(0.0, math.pi)
        off = rng.uniform(-1e-3, 1e-3, 2)
        depth = rng.uniform(0.1e-3, 1.0e-3)
        if kind == "sphere":
            params, tip = (rng.uniform(2e-3, 4e-3),), None
            tip = params[0]
        elif kind == "cylinder":
            params = (rng.uniform(1e-3, 2e-3), rng.uniform(2e-3, 4e-3))
            tip = params[0]
        elif kind == "cone":
            params, tip = (math.radians(rng.uniform(25.0, 45.0)), 3e-3), 0.0
        else:
            params, tip = (math.radians(rng.uniform(30.0, 60.0)), rng.uniform(1.5e-3, 3e-3), 3e-3), 0.0
        z_top = nz * C2_DX
        pose = (nx * C2_DX / 2 + off[0], ny * C2_DX / 2 + off[1], z_top + tip,
                math.cos(yaw / 2), 0.0, 0.0, math.sin(yaw / 2))
        out.append((blk, dict(kind=kind, params=params, pose=pose, depth=depth)))
    return out


# --------------------------------------------------------------------------
# Surrogate dataset (C3): presses of a C0-scale elastomer.
C3_BLOCK = Block(24, 24, 6, 0.5e-3, pad_side=4, pad_top=4)
C3_SUBSTEPS = 500
C3_DT = 1.0e-5
C3_SIZE = 64


def c3_specs(n, seed_base=0):
    """n random presses: an analytic indenter (sphere R U[2,4] mm, cylinder
    R U[1,2] mm x 8 mm, cone of half angle U[25,45] deg, prism of half angle
    U[30,60] deg x 8 mm), yaw U[0, pi), xy offset U[-1, 1] mm from the block
    centre, depth U[0.1, 1.0] mm; from numpy's PCG64 seeded with
    seed_base + i."""
    out = []
    b = C3_BLOCK
    for i in range(n):
        rng = np.random.default_rng(seed_base + i)
        kind = ["sphere", "cylinder", "cone", "prism"][int(rng.integers(4))]
        if kind == "sphere":
            params = (float(rng.uniform(2e-3, 4e-3)),)
            tip = params[0]
        elif kind == "cylinder":
            params = (float(rng.uniform(1e-3, 2e-3)), 4e-3)
            tip = params[0]
        elif kind == "cone":
            params, tip = (math.radians(float(rng.uniform(25.0, 45.0))), 3e-3), 0.0
        else:
            params, tip = (math.radians(float(rng.uniform(30.0, 60.0))), 4e-3, 3e-3), 0.0
        yaw = float(rng.uniform(0.0, math.pi))
        off = rng.uniform(-1e-3, 1e-3, 2)
        depth = float(rng.uniform(0.1e-3, 1.0e-3))
        z_top = b.nz * b.dx
        pose = (b.nx * b.dx / 2 + float(off[0]), b.ny * b.dx / 2 + float(off[1]), z_top + tip,
                math.cos(yaw / 2), 0.0, 0.0, math.sin(yaw / 2))
        out.append(dict(kind=kind, params=params, pose=pose, depth=depth, yaw=yaw, seed=seed_base + i))
    return out


# --------------------------------------------------------------------------
# Serving mix (C4): a Poisson stream of press queries on the C3 sensor.
def c4_queries(rate_hz=4096.0, duration_s=1.0, seed=4, out_of_range=0.10):
    """Arrival times (exponential gaps at rate_hz) and press specs: mostly
    presses like the training set; a fraction out of its range (depth 1.0-1.5
    mm, or a height-map dot-grid indenter the network never saw)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    i = 0
    while True:
        t += float(rng.exponential(1.0 / rate_hz))
        if t > duration_s:
            break
        spec = c3_specs(1, seed_base=10_000_000 + 97 * seed + i)[0]
        if rng.uniform() < out_of_range:
            if rng.uniform() < 0.5:
                spec["depth"] = float(rng.uniform(1.0e-3, 1.5e-3))
            else:
                b = C3_BLOCK
                hm = hm_dots(n=64, pix=0.1e-3, pitch=1.2e-3, count=4, height=0.8e-3)
                spec.update(kind="heightmap", params=(2e-3,), hm=hm,
                            pose=(b.nx * b.dx / 2, b.ny * b.dx / 2, b.nz * b.dx + float(hm.max()), 1.0, 0.0, 0.0, 0.0))
        spec["arrival"] = t
        spec["id"] = i
        out.append(spec)
        i += 1
    return out


def indenter_points(kind, params, n, seed=0, reach=1.0e-3):
    """n points sampled uniformly (numpy PCG64, seed) inside an analytic
    indenter, in its local frame (m), restricted to the part within `reach`
    of its lowest point (the part that can touch the elastomer): the point
    cloud of a particle-represented indenter.  Shapes and frames as in the
    C ABI: sphere (radius; centre at the origin), cylinder (radius, half
    length along local x; axis through the origin), cone (half angle,
    height; apex at the origin, opening to +z), prism (half angle, half
    length along local y, height; edge at the origin, opening to +z)."""
    rng = np.random.default_rng(seed)
    out = []
    while sum(len(o) for o in out) < n:
        m = 4 * n
        if kind == "sphere":
            R = params[0]
            p = rng.uniform([-R, -R, -R], [R, R, -R + reach], (m, 3))
            p = p[(p ** 2).sum(1) <= R * R]
        elif kind == "cylinder":
            R, L = params[0], params[1]
            p = rng.uniform([-L, -R, -R], [L, R, -R + reach], (m, 3))
            p = p[p[:, 1] ** 2 + p[:, 2] ** 2 <= R * R]
        elif kind == "cone":
            t = math.tan(params[0])
            h = min(params[1], reach)
            p = rng.uniform([-h * t, -h * t, 0.0], [h * t, h * t, h], (m, 3))
            p = p[np.hypot(p[:, 0], p[:, 1]) <= t * p[:, 2]]
        elif kind == "prism":
            t, L = math.tan(params[0]), params[1]
            h = min(params[2], reach)
            p = rng.uniform([-h * t, -L, 0.0], [h * t, L, h], (m, 3))
            p = p[np.abs(p[:, 0]) <= t * p[:, 2]]
        else:
            raise ValueError(kind)
        out.append(p)
    return np.concatenate(out)[:n]
