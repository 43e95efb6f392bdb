"""Serving a stream of press queries with the learned surrogate, falling back
to the batched MPM (this library's addition; the paper simulates one press at
a time).

Policy: queries are taken in windows; a query inside the surrogate's
training range (the trained sensor, shape families and depth range) is
answered by one batched network inference (up to max_batch per launch).
Other queries join the MPM lane, which runs as one batched MPM press when it
holds mpm_batch queries or its oldest query has waited mpm_wait_s (or the
stream ends), on pooled handles that are reset and reused.  Every
check_every-th in-range query also joins the MPM lane: if the surrogate
answer differs from the MPM's by more than residual_um (RMS of the vertical
displacement), the MPM answer is served instead, at the MPM lane's
completion time.  The clock is virtual and the GPU runs one lane at a time:
each batch of work advances the clock by its measured duration; latency =
completion - arrival.
"""
from __future__ import annotations

import time

import numpy as np

from . import IndenterKind, TacchiBatch, surrogate as SG

KINDS = {"sphere": IndenterKind.SPHERE, "cylinder": IndenterKind.CYLINDER, "cone": IndenterKind.CONE,
         "prism": IndenterKind.PRISM, "heightmap": IndenterKind.HEIGHTMAP}


def in_training_range(q):
    return q["kind"] in ("sphere", "cylinder", "cone", "prism") and 0.1e-3 <= q["depth"] <= 1.0e-3


class PressServer:
    def __init__(self, net, block, substeps, dt, size=64, max_batch=1024, check_every=64, residual_um=5.0,
                 use_surrogate=True, mpm_batch=256, mpm_wait_s=0.25, pool_sizes=(32, 128, 512, 1024)):
        import torch
        self.torch = torch
        self.net, self.block, self.substeps, self.dt, self.size = net, block, substeps, dt, size
        self.max_batch, self.check_every, self.residual_um = max_batch, check_every, residual_um
        self.use_surrogate = use_surrogate
        self.mpm_batch, self.mpm_wait_s = mpm_batch, mpm_wait_s
        self.pool_sizes = tuple(pool_sizes)
        self.pool = {}
        self.win = (0.0, 0.0, block.nx * block.dx, block.ny * block.dx)
        self.geo = TacchiBatch([block])  # geometry only: penetration maps of the query poses
        self.pen = torch.empty((size, size), device="cuda")
        self.X = torch.empty((max_batch, size, size, 2), device="cuda")
        self.Y = torch.empty((max_batch, size, size, 3), device="cuda")

    def _final_pose(self, q):
        p = list(q["pose"])
        p[2] -= q["depth"]
        return tuple(p)

    def _surrogate(self, qs):
        for i, q in enumerate(qs):
            self.geo.set_indenter(0, KINDS[q["kind"]], q["params"], self._final_pose(q), (0,) * 6)
            self.geo.penetration_map(0, self.size, self.size, self.win, out=self.pen)
            self.X[i, :, :, 0] = self.pen / SG.MM
            self.X[i, :, :, 1] = q["depth"] / SG.MM
        return self.net.forward(self.X[:len(qs)], out=self.Y[:len(qs)])

    def _handle(self, n):
        cap = next((c for c in self.pool_sizes if c >= n), self.pool_sizes[-1])
        if cap not in self.pool:
            self.pool[cap] = TacchiBatch([self.block] * cap)
        return self.pool[cap], cap

    def _mpm(self, qs):
        out = self.torch.empty((len(qs), self.size, self.size, 3), device="cuda")
        for c0 in range(0, len(qs), self.pool_sizes[-1]):
            part = qs[c0:c0 + self.pool_sizes[-1]]
            bt, cap = self._handle(len(part))
            bt.reset()
            for i in range(cap):
                if i < len(part):
                    q = part[i]
                    bt.set_indenter(i, KINDS[q["kind"]], q["params"], q["pose"],
                                    (0.0, 0.0, -q["depth"] / (self.substeps * self.dt), 0.0, 0.0, 0.0),
                                    hm=q.get("hm"), hm_pixel=0.1e-3)
                else:  # unused slot: no indenter, the sensor stays at rest
                    bt.set_indenter(i, IndenterKind.NONE, (), vel=(0,) * 6)
            bt.step(self.substeps, self.dt)
            if bt.status() != 0:
                raise RuntimeError("MPM fallback failed")
            for i in range(len(part)):
                bt.displacement_map(i, self.size, self.size, self.win, out=out[c0 + i])
        return out / SG.MM

    def serve(self, queries, window_s=0.02):
        torch = self.torch
        clock = 0.0
        lat = {}
        n_sur = n_check = n_reject = 0
        residuals = []
        pending = []  # MPM lane: (query, is_check, surrogate answer or None)
        k, nq = 0, len(queries)

        def run_mpm(now):
            nonlocal n_reject
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ref = self._mpm([p[0] for p in pending])
            for j, (q, is_check, pred) in enumerate(pending):
                if is_check:
                    r = float(torch.sqrt(((pred[..., 2] - ref[j, ..., 2]) * 1e3).pow(2).mean()))
                    residuals.append(r)
                    if r > self.residual_um:
                        n_reject += 1
                        pending[j] = (q, "served", None)
            torch.cuda.synchronize()
            now += time.perf_counter() - t0
            for q, flag, _ in pending:
                if flag is not True:  # fallback answers and replaced checks complete now
                    lat[q["id"]] = now - q["arrival"]
            pending.clear()
            return now

        while k < nq or pending:
            if k < nq:
                clock = max(clock, queries[k]["arrival"])
                end = clock + window_s
                batch = []
                while k < nq and queries[k]["arrival"] <= end and len(batch) < self.max_batch:
                    batch.append(queries[k])
                    k += 1
                # a full batch, or the end of the stream, starts at once; otherwise
                # the window closes first
                clock = max(clock, batch[-1]["arrival"]) if (len(batch) == self.max_batch or k == nq) else end
                sur = [q for q in batch if self.use_surrogate and in_training_range(q)]
                for q in batch:
                    if not (self.use_surrogate and in_training_range(q)):
                        pending.append((q, False, None))
                if sur:
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    pred = self._surrogate(sur)
                    torch.cuda.synchronize()
                    clock += time.perf_counter() - t0
                    n_sur += len(sur)
                    for i, q in enumerate(sur):
                        lat[q["id"]] = clock - q["arrival"]
                        if q["id"] % self.check_every == 0:
                            pending.append((q, True, pred[i].clone()))
                            n_check += 1
            oldest = min((p[0]["arrival"] for p in pending), default=None)
            if pending and (len(pending) >= self.mpm_batch or k == nq or clock - oldest >= self.mpm_wait_s):
                clock = run_mpm(clock)
        L = np.array([lat[q["id"]] for q in queries])
        n_fallback = sum(1 for q in queries if not (self.use_surrogate and in_training_range(q)))
        return {"queries": nq, "frames_per_s": nq / clock, "makespan_s": clock,
                "latency_p50_ms": float(np.percentile(L, 50) * 1e3),
                "latency_p99_ms": float(np.percentile(L, 99) * 1e3),
                "surrogate_answers": n_sur - n_reject, "mpm_answers": n_fallback + n_reject,
                "sampled_checks": n_check, "checks_over_residual": n_reject,
                "sampled_residual_um_mean": float(np.mean(residuals)) if residuals else None,
                "sampled_residual_um_p99": float(np.percentile(residuals, 99)) if residuals else None}
