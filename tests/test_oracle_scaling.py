"""Pins of the paper's printed numbers: Table 1 from Eq. 8, the Re worked
example of Sec. 3.3, the uniformity measures of Eq. 9-11."""
import math
import os

import numpy as np
import pytest

from oracle import scaling

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            rows.append([float(v) for v in line.split()])
    return rows


def test_eq8_reproduces_table1():
    table = {int(s): w for s, w in _rows("table1_widths.txt")}
    widths = scaling.eq8_widths(w_smallest=table[4], h=10.0, scales=4)  # [w4, w3, w2, w1]
    for scale, w in zip((4, 3, 2, 1), widths):
        assert w == pytest.approx(table[scale], rel=0.01), (scale, w)
    # each consecutive pair satisfies Eq. 8 itself
    for small, large in zip(widths[:-1], widths[1:]):
        assert abs(scaling.eq8_residual(small, large, 10.0)) < 1e-12
    # ratio close to 0.68-0.69 as the text implies
    assert all(0.66 < a / b < 0.70 for a, b in zip(widths[:-1], widths[1:]))


def test_eq8_limit_of_deep_channels():
    # h -> 0: (w_{k+1}/w_k)^4 * w_k^2 / w_{k+1}^2 = 1/4  ->  ratio = 1/2 exactly
    w = scaling.eq8_next_wider(1.0, h=1e-12)
    assert w == pytest.approx(2.0, rel=1e-9)
    # h -> infinity: (w_{k+1}/w_k)^4 = 1/4  ->  ratio = 2^(-1/2)
    w = scaling.eq8_next_wider(1.0, h=1e9)
    assert w == pytest.approx(math.sqrt(2.0), rel=1e-6)


def test_reynolds_worked_example():
    (w_in, u_in, nu, re), = _rows("reynolds_example.txt")
    assert scaling.reynolds(w_in, u_in, nu) == pytest.approx(re, rel=1e-12)
    # nu = 0.04 <-> tau = 3 nu + 1/2 = 0.62
    assert scaling.viscosity(0.62) == pytest.approx(0.04, rel=1e-12)


def test_uniformity_closed_forms(ora):
    th, dg = ora.uniformity([2.0, 2.0, 2.0, 2.0])
    assert th == 1.0 and dg == 0.0
    th, dg = ora.uniformity([1.0, 2.0])
    assert th == 2.0
    assert dg == pytest.approx(math.sqrt(2.0) / 3.0, rel=1e-15)
    m = np.array([0.9, 1.1, 1.0, 1.05, 0.95])
    th, dg = ora.uniformity(m)
    ave = m.mean()
    assert th == pytest.approx(1.1 / 0.9, rel=1e-15)
    assert dg == pytest.approx(math.sqrt(((m / ave - 1) ** 2).sum() / 4), rel=1e-14)
    # D_g is scale-free: scaling all flow rates leaves it unchanged
    th2, dg2 = ora.uniformity(7.0 * m)
    assert dg2 == pytest.approx(dg, rel=1e-13) and th2 == pytest.approx(th, rel=1e-14)
