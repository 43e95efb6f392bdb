"""Serving a stream of press queries with the learned surrogate, falling back
to the batched MPM (this library's addition; the paper simulates one press at
a time).

Policy: a query inside the surrogate's range (the trained sensor, shape
families and depth range, or a narrower validity region calibrated on
held-out presses) is answered by one batched network inference
(up to max_batch queries per launch) as soon as the server looks at it.
Other queries join the MPM lane, which starts a batched MPM press (on pooled
handles that are reset and reused) when it holds mpm_batch queries, its
oldest query has waited mpm_wait_s, or the stream ends.  The press advances
in chunks of chunk_substeps substeps, and arrived queries are answered by the
surrogate between chunks, so the network lane is not held up by the MPM.
Every check_every-th in-range query also joins the MPM lane: if the surrogate
answer differs from the MPM's by more than residual_um (RMS of the vertical
displacement), the MPM answer is served instead, at the press's completion.
The clock is virtual: the GPU does one piece of work at a time and each piece
advances the clock by its measured duration; latency = completion - arrival.
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
                 use_surrogate=True, mpm_batch=256, mpm_wait_s=0.25, pool_sizes=(32, 128, 512, 1024),
                 in_range=None):
        import torch
        self.torch = torch
        self._policy(substeps, dt, size, max_batch, check_every, residual_um, use_surrogate, mpm_batch,
                     mpm_wait_s, pool_sizes, in_range)
        self.net, self.block = net, block
        self.pool = {}
        self.win = (0.0, 0.0, block.nx * block.dx, block.ny * block.dx)
        self.geo = TacchiBatch([block])  # geometry only: penetration maps of the query poses
        self.pen = torch.empty((size, size), device="cuda")
        self.X = torch.empty((max_batch, size, size, 2), device="cuda")
        self.Y = torch.empty((max_batch, size, size, 3), device="cuda")

    def _policy(self, substeps, dt, size, max_batch, check_every, residual_um, use_surrogate, mpm_batch,
                mpm_wait_s, pool_sizes, in_range=None):
        # which queries the surrogate may answer: the training range, or a
        # validity region calibrated on held-out presses (surrogate.calibrate_region)
        self.in_range = in_range or in_training_range
        self.substeps, self.dt, self.size = substeps, dt, size
        self.max_batch, self.check_every, self.residual_um = max_batch, check_every, residual_um
        self.use_surrogate = use_surrogate
        self.mpm_batch, self.mpm_wait_s = mpm_batch, mpm_wait_s
        self.pool_sizes = tuple(pool_sizes)

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

    def _start_press(self, qs):
        bt, cap = self._handle(len(qs))
        bt.reset()
        for i in range(cap):
            if i < len(qs):
                q = qs[i]
                bt.set_indenter(i, KINDS[q["kind"]], q["params"], q["pose"],
                                (0.0, 0.0, -q["depth"] / (self.substeps * self.dt), 0.0, 0.0, 0.0),
                                hm=q.get("hm"), hm_pixel=0.1e-3)
            else:  # unused slot: no indenter, the sensor stays at rest
                bt.set_indenter(i, IndenterKind.NONE, (), vel=(0,) * 6)
        return {"handle": bt, "left": self.substeps}

    # -- device work, each timed by _run -----------------------------------------
    def _run(self, fn):
        """Runs fn on the device; returns its result and its duration (s)."""
        torch = self.torch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    def _advance(self, job, n):
        job["handle"].step(n, self.dt)

    def _finish(self, job):
        """Displacement maps (mm) of a completed press, one per query."""
        bt, n = job["handle"], len(job["items"])
        if bt.status() != 0:
            raise RuntimeError("MPM press failed")
        out = self.torch.empty((n, self.size, self.size, 3), device="cuda")
        for i in range(n):
            bt.displacement_map(i, self.size, self.size, self.win, out=out[i])
        return out / SG.MM

    def _residual_um(self, pred, ref):
        """RMS difference of the vertical displacement, um (maps in mm)."""
        return float(self.torch.sqrt(((pred[..., 2] - ref[..., 2]) * 1e3).pow(2).mean()))

    # -- the dispatcher -----------------------------------------------------------
    def serve(self, queries, chunk_substeps=50):
        clock = 0.0
        lat = {}
        n_sur = n_check = n_reject = 0
        residuals = []
        pending = []   # waiting for the MPM lane: (query, surrogate answer if a check)
        job = None     # running MPM press: handle, substeps left, its queries
        presses = []   # queries per MPM press
        mpm_served = []
        k, nq = 0, len(queries)

        def timed(fn):
            nonlocal clock
            out, sec = self._run(fn)
            clock += sec
            return out

        while k < nq or pending or job:
            if k < nq and queries[k]["arrival"] <= clock:
                batch = []
                while k < nq and queries[k]["arrival"] <= clock and len(batch) < self.max_batch:
                    batch.append(queries[k])
                    k += 1
                sur = [q for q in batch if self.use_surrogate and self.in_range(q)]
                pending += [(q, None) for q in batch if not (self.use_surrogate and self.in_range(q))]
                if sur:
                    pred = timed(lambda: self._surrogate(sur))
                    n_sur += len(sur)
                    for i, q in enumerate(sur):
                        lat[q["id"]] = clock - q["arrival"]
                        if q["id"] % self.check_every == 0:
                            pending.append((q, pred[i].clone()))
                            n_check += 1
            elif job is not None:
                n = min(chunk_substeps, job["left"])
                timed(lambda: self._advance(job, n))
                job["left"] -= n
                if job["left"] == 0:
                    ref = timed(lambda: self._finish(job))
                    for j, (q, pred) in enumerate(job["items"]):
                        if pred is None:
                            lat[q["id"]] = clock - q["arrival"]
                            mpm_served.append(q["id"])
                        else:
                            r = self._residual_um(pred, ref[j])
                            residuals.append(r)
                            if r > self.residual_um:  # the MPM answer is served instead
                                n_reject += 1
                                lat[q["id"]] = clock - q["arrival"]
                                mpm_served.append(q["id"])
                    job = None
            elif pending and (len(pending) >= self.mpm_batch or k == nq or
                              clock >= min(p[0]["arrival"] for p in pending) + self.mpm_wait_s):
                items = pending[:self.pool_sizes[-1]]
                pending = pending[len(items):]
                job = timed(lambda: self._start_press([p[0] for p in items]))
                job["items"] = items
                presses.append(len(items))
            else:
                nxt = queries[k]["arrival"] if k < nq else float("inf")
                if pending:
                    nxt = min(nxt, min(p[0]["arrival"] for p in pending) + self.mpm_wait_s)
                clock = max(clock, nxt)
        def pct(ids, q):
            x = [lat[i] for i in ids]
            return float(np.percentile(x, q) * 1e3) if x else None

        all_ids = [q["id"] for q in queries]
        by_mpm = set(mpm_served)
        sur_ids = [i for i in all_ids if i not in by_mpm]
        n_fallback = sum(1 for q in queries if not (self.use_surrogate and self.in_range(q)))
        return {"queries": nq, "frames_per_s": nq / clock if clock > 0 else 0.0, "makespan_s": clock,
                "latency_p50_ms": pct(all_ids, 50), "latency_p99_ms": pct(all_ids, 99),
                "latency_surrogate_p99_ms": pct(sur_ids, 99), "latency_mpm_p99_ms": pct(list(by_mpm), 99),
                "surrogate_answers": n_sur - n_reject, "mpm_answers": n_fallback + n_reject,
                "mpm_presses": presses,
                "sampled_checks": n_check, "checks_over_residual": n_reject,
                "sampled_residual_um_mean": float(np.mean(residuals)) if residuals else None,
                "sampled_residual_um_p99": float(np.percentile(residuals, 99)) if residuals else None}
