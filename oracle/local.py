"""Substeps of the method in FP64 over the particles of one box of grid
nodes, from the oracle's per-particle routines (B-spline weights, polar
decomposition and stress): P2G (Eqs. 2-5), grid velocity (Eq. 6), G2P, the
F update and advection (Eqs. 7-11).

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
    V = np.zeros_like(MG)
    pos = M > 0
    V[pos] = MG[pos] / M[pos][:, None]
    return V
