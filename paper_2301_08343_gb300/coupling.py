"""Coupling with a main (robot) simulator (Sec. III-C, Fig. 3).

Every simulation step the main simulator moves the objects; Tacchi takes the
indenter's motion -- a pose (position-driven, as with Gazebo) or a velocity
(velocity-driven, as with MuJoCo) -- advances the elastomer under it for one
frame of substeps (Eq. 11 moves the rigid indenter), and renders the depth
map and tactile image (Sec. III-B).  A terminal condition, checked on either
side, ends the episode (for example the indenter, or the surface it pushes,
reaching a desired depth).

There is no robot simulator in this package; `Coupler` is the loop on the
Tacchi side, driven by any source of poses or velocities (a recorded
trajectory in the tests).
"""
from __future__ import annotations

import math

import numpy as np


def _qmul(a, b):
    return (a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3],
            a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2],
            a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1],
            a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0])


def velocity_between(pose_a, pose_b, duration):
    """Constant twist (v, w) that carries pose_a to pose_b in `duration`
    seconds: v = (p_b - p_a) / T; w = axis * angle / T of the rotation
    q_b q_a^-1 (shortest way).  Poses are (x, y, z, qw, qx, qy, qz)."""
    v = [(pose_b[a] - pose_a[a]) / duration for a in range(3)]
    qa = np.asarray(pose_a[3:], np.float64)
    qb = np.asarray(pose_b[3:], np.float64)
    qa = qa / np.linalg.norm(qa)
    qb = qb / np.linalg.norm(qb)
    r = np.asarray(_qmul(qb, (qa[0], -qa[1], -qa[2], -qa[3])))
    if r[0] < 0:
        r = -r
    s = math.sqrt(max(0.0, 1.0 - min(1.0, r[0]) ** 2))
    angle = 2.0 * math.atan2(s, r[0])
    axis = r[1:] / s if s > 1e-300 else np.zeros(3)
    w = axis * angle / duration
    return (*v, *w)


class Coupler:
    """Tacchi's side of the loop of Fig. 3 for one sensor (a `Tacchi`).

    frame: one step of the main simulator = `substeps` substeps of `dt`.
    Each call of `step_pose` / `step_velocity` advances one frame and returns
    the frame's record: the indenter pose, the tactile image and depth map
    (device tensors) and the surface indentation (m, the largest depression
    of the rendered depth map below the rest top face)."""

    def __init__(self, sim, substeps, dt, size=(320, 240), window=None, rp=None):
        self.sim, self.substeps, self.dt = sim, int(substeps), float(dt)
        self.w, self.h = size
        self.window = window
        self.rp = rp
        self.frames = 0

    def _frame(self):
        import torch
        H = torch.empty((self.h, self.w), device=self.sim.device)
        img = self.sim.render(self.w, self.h, self.window, self.rp, out_height=H)
        depth = float(self.sim.z_top - H.min())
        self.frames += 1
        return {"frame": self.frames, "pose": self.sim.indenter_pose(), "image": img, "height": H,
                "surface_depth": depth, "status": self.sim.status()}

    def step_velocity(self, vel):
        """Velocity-driven: the indenter moves with twist `vel` for one frame."""
        self.sim.set_indenter(vel=tuple(float(x) for x in vel))
        self.sim.step(self.substeps, self.dt)
        return self._frame()

    def step_pose(self, pose):
        """Position-driven: the indenter reaches `pose` at the end of the
        frame, moving with the constant twist that gets it there."""
        vel = velocity_between(self.sim.indenter_pose(), pose, self.substeps * self.dt)
        return self.step_velocity(vel)

    def run(self, commands, terminal, mode="pose"):
        """Drive the loop with a sequence of poses (mode "pose") or twists
        (mode "velocity") until `terminal(record)` is true or the commands
        run out; returns the list of frame records."""
        out = []
        for cmd in commands:
            rec = self.step_pose(cmd) if mode == "pose" else self.step_velocity(cmd)
            out.append(rec)
            if rec["status"] != 0 or terminal(rec):
                break
        return out
