"""The Hertz contact law on the oracle: a = sqrt(R d), required within 5%.

oracle/hertz.py presses a rigid sphere (R = 6 mm) quasi-statically into a
14 x 14 x 7 mm block at dX = 0.1 mm with every step of the oracle's method
(about 5.5e10 particle-substeps, hours of host time) and stores the binned
top-surface profile at four depths in tests/golden/hertz_oracle.json.  Here
the profile is fitted with Hertz's half-space solution (d and a free, R not
used), a^2 = k d is fitted through the origin over the depths, and
|k / R - 1| <= 5% is required.  The stored profile belongs to one version of
the oracle: its source hash must match the current oracle, so that a change
to the oracle's arithmetic forces the run to be repeated."""
import json
import math
import os

import numpy as np
import pytest

from hertz_fit import fit_profile, hertz_shape, k_over_R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hertz_oracle.json")


def test_hertz_fit_recovers_its_own_profile():
    r = np.linspace(0.0, 4e-3, 400)
    a, d = 1.5e-3, 1.5e-3 ** 2 / 6e-3
    af, df = fit_profile(r, d * hertz_shape(r / a), 1.2e-3)
    assert af == pytest.approx(a, rel=2e-3) and df == pytest.approx(d, rel=2e-3)


def test_oracle_meets_the_hertz_contact_law():
    from oracle import hertz
    with open(GOLDEN) as f:
        ref = json.load(f)
    assert ref["oracle_sha1"] == hertz.source_hash(), "the oracle changed: rerun python -m oracle.hertz"
    cfg = ref["config"]
    assert ref["particles"] == 8 * cfg["nx"] ** 2 * cfg["nz"]
    R = cfg["R"]
    r = np.array(ref["r_m"])
    fits = []
    for prof in ref["profiles"]:
        d, w = prof["depth_m"], np.array(prof["w_m"])
        a, dfit = fit_profile(r, w, math.sqrt(R * d))
        fits.append((d, a, dfit))
        # the surface under the indenter follows it to within the grid
        # boundary's offset of about one node spacing
        assert 0.8 * d <= dfit <= 1.0 * d, (d, dfit)
        assert w[0] > w[-1] >= -0.05 * d  # deepest on the axis, flat far out
    assert np.all(np.diff([f[1] for f in fits]) > 0)
    assert abs(k_over_R(fits, R) - 1.0) <= 0.05, (k_over_R(fits, R), fits)
