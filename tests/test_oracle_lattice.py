"""Pins of the oracle's lattice tables and equilibrium (Sec. 2.1).

The velocity set is checked against the paper's cos/sin formula for the axis
directions, the weights against the printed fractions (golden file), and the
equilibrium against the moment identities that any correct second-order D2Q9
f^eq must satisfy -- a dropped term, a wrong sign or a wrong bracket in the
second-order term breaks the second moment.
"""
import math
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_weights():
    w, cs2, speed2 = {}, None, {}
    for line in open(os.path.join(GOLDEN, "d2q9_constants.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        parts = line.split()
        if parts[0] == "cs2":
            cs2 = Fraction(int(parts[1]), int(parts[2]))
        else:
            w[int(parts[0])] = Fraction(int(parts[1]), int(parts[2]))
            speed2[int(parts[0])] = int(parts[3])
    return w, cs2, speed2


def test_axis_directions_follow_printed_formula(ora):
    cx, cy, opp, w, cs2 = ora.lattice()
    for i in range(1, 5):
        ang = (i - 1) * math.pi / 2
        assert (cx[i], cy[i]) == (round(math.cos(ang)), round(math.sin(ang)))
    assert (cx[0], cy[0]) == (0, 0)


def test_diagonals_standard_reading(ora):
    # the printed diagonal formula (length sqrt2, angle (i-5)pi/2) is garbled;
    # the reading is angle (i-5)pi/2 + pi/4 at length sqrt2
    cx, cy, *_ = ora.lattice()
    for i in range(5, 9):
        ang = (i - 5) * math.pi / 2 + math.pi / 4
        assert (cx[i], cy[i]) == (round(math.sqrt(2) * math.cos(ang)), round(math.sqrt(2) * math.sin(ang)))


def test_weights_and_sound_speed_match_paper(ora):
    cx, cy, opp, w, cs2 = ora.lattice()
    gw, gcs2, speed2 = _golden_weights()
    for i in range(9):
        assert w[i] == float(gw[i])
        assert cx[i] ** 2 + cy[i] ** 2 == speed2[i]
    assert cs2 == float(gcs2)


def test_opposites(ora):
    cx, cy, opp, *_ = ora.lattice()
    for i in range(9):
        assert cx[opp[i]] == -cx[i] and cy[opp[i]] == -cy[i]
        assert opp[opp[i]] == i


def test_lattice_isotropy_exact(ora):
    """sum w = 1, sum w c = 0, sum w c_a c_b = c_s^2 delta_ab, 4th moment isotropic (exact rationals)."""
    cx, cy, opp, w, cs2 = ora.lattice()
    gw, gcs2, _ = _golden_weights()
    W = [gw[i] for i in range(9)]
    assert sum(W) == 1
    assert sum(W[i] * int(cx[i]) for i in range(9)) == 0
    assert sum(W[i] * int(cy[i]) for i in range(9)) == 0
    assert sum(W[i] * int(cx[i]) ** 2 for i in range(9)) == gcs2
    assert sum(W[i] * int(cy[i]) ** 2 for i in range(9)) == gcs2
    assert sum(W[i] * int(cx[i]) * int(cy[i]) for i in range(9)) == 0
    # fourth moment: sum w c_x^2 c_y^2 = c_s^4 and sum w c_x^4 = 3 c_s^4
    assert sum(W[i] * int(cx[i]) ** 2 * int(cy[i]) ** 2 for i in range(9)) == gcs2 ** 2
    assert sum(W[i] * int(cx[i]) ** 4 for i in range(9)) == 3 * gcs2 ** 2


def test_feq_moments(ora):
    """sum f^eq = rho, sum c f^eq = rho u, sum c c f^eq = rho c_s^2 I + rho u u."""
    cx, cy, *_ = ora.lattice()
    rng = np.random.default_rng(7)
    for _ in range(50):
        rho = 0.5 + rng.random()
        ux, uy = 0.2 * (rng.random(2) - 0.5)
        f = np.array([ora.feq(i, rho, ux, uy) for i in range(9)])
        assert abs(f.sum() - rho) <= 1e-15 * 4
        assert abs((cx * f).sum() - rho * ux) <= 1e-15 * 4
        assert abs((cy * f).sum() - rho * uy) <= 1e-15 * 4
        pxx = (cx * cx * f).sum()
        pyy = (cy * cy * f).sum()
        pxy = (cx * cy * f).sum()
        assert abs(pxx - (rho / 3 + rho * ux * ux)) <= 1e-15 * 4
        assert abs(pyy - (rho / 3 + rho * uy * uy)) <= 1e-15 * 4
        assert abs(pxy - rho * ux * uy) <= 1e-15 * 4


def test_feq_at_rest_is_weighted_density(ora):
    cx, cy, opp, w, cs2 = ora.lattice()
    for i in range(9):
        assert ora.feq(i, 1.25, 0.0, 0.0) == w[i] * 1.25
