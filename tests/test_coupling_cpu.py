"""Host side of the loop with a main simulator (Sec. III-C): the constant
twist that carries one pose to the next.  Checked against closed forms and by
integrating the twist back with small rotation steps (a rotation about a
fixed world axis composes exactly, so many small steps land on the target)."""
import math

import numpy as np

from paper_2301_08343_gb300.coupling import velocity_between


def qmul(a, b):
    return np.array([a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3],
                     a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2],
                     a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1],
                     a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0]])


def integrate(pose, twist, T, n):
    p = np.array(pose[:3], float)
    q = np.array(pose[3:], float)
    w = np.array(twist[3:], float)
    for _ in range(n):
        p += np.array(twist[:3]) * (T / n)
        wn = np.linalg.norm(w)
        if wn > 0:
            h = 0.5 * wn * T / n
            q = qmul(np.concatenate([[math.cos(h)], math.sin(h) * w / wn]), q)
    return p, q


def test_yaw_about_z_closed_form():
    a = (0.001, 0.002, 0.003, math.cos(0.1), 0.0, 0.0, math.sin(0.1))
    ang = 0.3
    b = (0.002, 0.002, 0.001, math.cos(0.1 + ang / 2), 0.0, 0.0, math.sin(0.1 + ang / 2))
    v = velocity_between(a, b, 0.5)
    assert np.allclose(v, (0.002, 0.0, -0.004, 0.0, 0.0, ang / 0.5), atol=1e-12)


def test_no_motion_is_zero_twist_and_sign_of_q_does_not_matter():
    a = (0.0, 0.0, 0.0, 0.6, 0.0, 0.8, 0.0)
    assert np.allclose(velocity_between(a, a, 1.0), 0.0, atol=1e-12)
    b = tuple(-x for x in a[3:])
    assert np.allclose(velocity_between(a, (0.0, 0.0, 0.0) + b, 1.0), 0.0, atol=1e-12)


def test_general_rotation_integrates_back_to_the_target():
    rng = np.random.default_rng(4)
    for _ in range(20):
        qa = rng.normal(size=4)
        qa /= np.linalg.norm(qa)
        qb = rng.normal(size=4)
        qb /= np.linalg.norm(qb)
        a = tuple(rng.normal(size=3)) + tuple(qa)
        b = tuple(rng.normal(size=3)) + tuple(qb)
        T = float(rng.uniform(0.1, 2.0))
        tw = velocity_between(a, b, T)
        # the shortest way: the turned angle is at most pi
        assert np.linalg.norm(tw[3:]) * T <= math.pi + 1e-12
        p, q = integrate(a, tw, T, 64)
        assert np.allclose(p, b[:3], atol=1e-12)
        assert abs(abs(float(q @ qb)) - 1.0) < 1e-12
