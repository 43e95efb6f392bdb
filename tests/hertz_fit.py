"""Hertz contact of a rigid sphere on an elastic half-space (Hertz 1882;
Johnson, Contact Mechanics, Sec. 4.2): contact radius a with a^2 = R d, and
the vertical surface displacement
    w(r) = d (1 - rho^2 / 2)                                         rho <= 1,
    w(r) = (d / pi) ((2 - rho^2) asin(1 / rho) + sqrt(rho^2 - 1))    rho > 1,
with rho = r / a.  A measured profile gives d and a by least squares over
r <= 2 a; the sphere's radius is not used, so a^2 = k d fitted over several
depths tests the law through k / R."""
import numpy as np


def hertz_shape(rho):
    rho = np.asarray(rho, float)
    out = np.where(rho <= 1.0, 1.0 - rho ** 2 / 2.0, 0.0)
    m = rho > 1.0
    r = rho[m]
    out[m] = ((2.0 - r ** 2) * np.arcsin(1.0 / r) + np.sqrt(r ** 2 - 1.0)) / np.pi
    return out


def fit_profile(r, w, a_guess):
    """Least-squares (d, a) of w ~ d h(r / a) over r <= 2 a (scan of a, d in
    closed form)."""
    best = None
    for a in np.linspace(0.6 * a_guess, 1.6 * a_guess, 801):
        m = r <= 2.0 * a
        h = hertz_shape(r[m] / a)
        d = float(h @ w[m]) / float(h @ h)
        res = float(((d * h - w[m]) ** 2).mean())
        if best is None or res < best[0]:
            best = (res, a, d)
    return best[1], best[2]


def k_over_R(fits, R):
    """Slope k of a^2 = k d through the origin over (depth, a, d) fits, / R."""
    a = np.array([f[1] for f in fits])
    d = np.array([f[2] for f in fits])
    return float((a ** 2) @ d / (d @ d)) / R
