"""Substeps of the method in FP64 over the particles of one box of grid
nodes, from the oracle's per-particle routines (B-spline weights, polar
decomposition and stress): P2G (Eqs. 2-5), grid velocity (Eq. 6) with the
indenter, base and padding-band conditions, G2P, the F update and advection
(Eqs. 7-11).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the full-size sampled
parity tests recompute two substeps around sampled grid nodes with it, where
the whole-grid oracle would take hours.  Pinned against the oracle's own
whole-grid substeps (tests/test_sampled_mpm_cpu.py) and against an affine
grid velocity field, which Eqs. 7-9 reproduce exactly
(tests/test_oracle_pins.py)."""
import numpy as np

from . import stress as _stress
from . import weights as _weights


class Local:
    """Substeps of the method in FP64 over the particles of one box."""

    def __init__(self, dx, dt, E, nu, rho):
        self.dx, self.dt = dx, dt
        self.mu = E / (2 * (1 + nu))
        self.la = E * nu / ((1 + nu) * (1 - 2 * nu))
        self.V0 = dx ** 3 / 8
        self.m = rho * self.V0

    def weights(self, u):
        base = np.zeros((len(u), 3), np.int64)
        w = np.zeros((len(u), 3, 3, 3))
        for p in range(len(u)):
            b, wp = _weights(u[p])
            base[p], w[p] = b, wp
        return base, w  # w[p][k][j][i]

    def p2g(self, u, v, C, F, lo, shape):
        """(M, MG) on nodes lo + [0, shape) from every given particle."""
        base, w = self.weights(u)
        tau = np.stack([_stress(F[p], self.mu, self.la) for p in range(len(u))])
        A = self.m * C - self.dt * self.V0 * 4.0 / self.dx ** 2 * tau
        M = np.zeros(shape)
        MG = np.zeros(shape + (3,))
        for k in range(3):
            for j in range(3):
                for i in range(3):
                    node = base + np.array([i, j, k])
                    d = (node - u) * self.dx                       # X_i - x_p (m)
                    wk = w[:, k, j, i]
                    mom = wk[:, None] * (self.m * v + np.einsum("pab,pb->pa", A, d))
                    idx = tuple((node - lo).T[::-1])                 # [z][y][x]
                    np.add.at(M, idx, wk * self.m)
                    np.add.at(MG, idx, mom)
        return M, MG

    def g2p(self, u, F, fixed, V, lo):
        """Eqs. 7-11 with the grid velocity V on nodes lo + [0, shape)."""
        base, w = self.weights(u)
        v = np.zeros((len(u), 3))
        B = np.zeros((len(u), 3, 3))
        for k in range(3):
            for j in range(3):
                for i in range(3):
                    node = base + np.array([i, j, k])
                    Vi = V[tuple((node - lo).T[::-1])]
                    wk = w[:, k, j, i]
                    v += wk[:, None] * Vi
                    B += wk[:, None, None] * np.einsum("pa,pb->pab", Vi, (node - u) * self.dx)
        C = 4.0 / self.dx ** 2 * B
        F = np.einsum("pab,pbc->pac", np.eye(3)[None] + self.dt * C, F)
        v[fixed] = 0.0
        u = u + self.dt / self.dx * v
        return u, v, C, F


def velocity(M, MG):
    """Eq. 6 alone: V = MG / M where M > 0, else 0."""
    V = np.zeros_like(MG)
    pos = M > 0
    V[pos] = MG[pos] / M[pos][:, None]
    return V


def grid_velocity(M, MG, lo, G, dx=None, origin=None, inside=None, pose=None, vel=None, base_k=None):
    """Eq. 6 and the boundary conditions over the box's nodes lo + [0, shape),
    in the order of the oracle's grid update: a node inside the indenter
    (inside(i, j, k), the oracle's own decision at the pose of the substep)
    takes the indenter's rigid velocity v + w x (X - c) (Eq. 10); a node at or
    below the base layer base_k takes 0 (the fixed base, Eq. 10); the outer
    two node layers of the grid (G nodes per axis) take 0."""
    V = velocity(M, MG)
    nz, ny, nx = M.shape
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                I, J, K = lo[0] + i, lo[1] + j, lo[2] + k
                if inside is not None and inside(I, J, K):
                    r = origin + dx * np.array([I, J, K], float) - np.asarray(pose[:3], float)
                    V[k, j, i] = np.asarray(vel[:3], float) + np.cross(np.asarray(vel[3:], float), r)
                if base_k is not None and K <= base_k:
                    V[k, j, i] = 0.0
                if I < 2 or J < 2 or K < 2 or I > G[0] - 3 or J > G[1] - 3 or K > G[2] - 3:
                    V[k, j, i] = 0.0
    return V
