"""The Hertz contact law on the oracle: a rigid sphere pressed quasi-statically
into the elastomer, the top-surface profile recorded at four depths.

TEST INFRASTRUCTURE ONLY.  Writes tests/golden/hertz_oracle.json, which
tests/test_oracle_hertz.py fits: a sphere of radius R pressed a depth d into
an elastic half-space touches it over a disc of radius a with a^2 = R d
(Hertz 1882; Johnson, Contact Mechanics, Sec. 4.2).

Setup (FP64 oracle, every step of Sec. III-A): a 14 x 14 x 7 mm block at
dX = 0.1 mm (140 x 140 x 70 cells, 10,976,000 particles, lattice seed 1),
E 0.3 MPa, nu 0.45, rho 1000, fixed base; a sphere of R = 6 mm over the block
centre, tangent to the top face, pressed at 0.1 m/s with dt = 2e-6 s to the
depths 0.3, 0.4, 0.5, 0.6 mm, each followed by a 500-substep hold; the
vertical displacement of every top-layer particle is averaged over the last
250 substeps of each hold (five samples 50 substeps apart) and binned by its
rest distance from the axis (bins of dX / 4).  About 5.5e10 particle-substeps:
hours on a many-core host.

  python -m oracle.hertz [--threads N] [--out tests/golden/hertz_oracle.json]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import time

import numpy as np

from . import IND_SPHERE, Sim, lattice, set_threads

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CONFIG = dict(nx=140, nz=70, dx=0.1e-3, E=3.0e5, nu=0.45, rho=1000.0, seed=1, R=6e-3, speed=0.1, dt=2e-6,
              depths=[0.3e-3, 0.4e-3, 0.5e-3, 0.6e-3], hold=500, average=250, sample_every=50)


def source_hash():
    """SHA-1 of the oracle's C source: a stored profile is valid for it only."""
    h = hashlib.sha1()
    for name in ("tacchi_oracle.c", "tacchi_oracle.h"):
        with open(os.path.join(HERE, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def run(cfg=CONFIG, threads=None, log=print):
    set_threads(threads or os.cpu_count() or 1)
    nx, nz, dx = cfg["nx"], cfg["nz"], cfg["dx"]
    s = Sim(nx, nx, nz, dx, cfg["E"], cfg["nu"], cfg["rho"])
    u0, fl = lattice(nx, nx, nz, 4, 3, cfg["seed"])
    s.set_state(u0, flags=fl)
    s.set_rest(u0)
    top = (fl & 2) > 0
    c = nx * dx / 2
    xr = s.origin[:2, None] + u0[:2, top].astype(np.float64) * dx
    r = np.hypot(xr[0] - c, xr[1] - c)
    bw = dx / 4
    nb = int(3.5e-3 / bw)
    idx = np.minimum((r / bw).astype(int), nb)
    keep = [i for i in range(nb) if np.any(idx == i)]
    rb = [float(r[idx == i].mean()) for i in keep]
    R, v, dt = cfg["R"], cfg["speed"], cfg["dt"]
    s.set_indenter(IND_SPHERE, (R,), (c, c, s.z_top + R, 1.0, 0.0, 0.0, 0.0), (0.0, 0.0, -v, 0.0, 0.0, 0.0))
    cur, out, t0 = 0.0, [], time.time()
    for d in cfg["depths"]:
        n = int(round((d - cur) / (v * dt)))
        s.set_indenter(IND_SPHERE, (R,), tuple(s.pose()), (0.0, 0.0, -v, 0.0, 0.0, 0.0))
        err = s.run(n, dt)
        cur += n * v * dt
        s.set_indenter(IND_SPHERE, (R,), tuple(s.pose()), (0.0, 0.0, 0.0, 0.0, 0.0, 0.0))
        err |= s.run(cfg["hold"] - cfg["average"], dt)
        ws = []
        for _ in range(cfg["average"] // cfg["sample_every"]):
            err |= s.run(cfg["sample_every"], dt)
            xi = s.state()[0]
            ws.append(-(xi[2, top] - u0[2, top].astype(np.float64)) * dx)
        if err:
            raise RuntimeError(f"oracle error bits {err} at depth {d}")
        w = np.mean(ws, axis=0)
        out.append({"depth_m": cur, "w_m": [float(w[idx == i].mean()) for i in keep]})
        log(f"depth {cur * 1e3:.3f} mm done after {time.time() - t0:.0f} s")
    return {"config": cfg, "r_m": rb, "profiles": out, "oracle_sha1": source_hash(),
            "particles": int(s.N), "seconds": time.time() - t0, "threads": threads or os.cpu_count()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--out", default=os.path.join(ROOT, "tests", "golden", "hertz_oracle.json"))
    a = ap.parse_args()
    res = run(threads=a.threads or None, log=lambda m: print(m, flush=True))
    with open(a.out, "w") as f:
        json.dump(res, f, indent=1)
    print("wrote", a.out)


if __name__ == "__main__":
    main()
