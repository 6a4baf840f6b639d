"""Pins of the oracle's convergence residual (Sec. 2.3 step 5: the "exact flow
field" of step 2 is a converged solve; the residual reported with every solve
is r = sum |u(T) - u(T-K)|_1 / sum |u(T)|_1 over the fluid cells, K = 100).

Each check is fixed by something other than the oracle:
  * a field small enough to work out by hand (below), where the L1 ratio,
    an L2 ratio, a ratio without the absolute values and a ratio that counts
    solid cells all differ;
  * the closed form of a decaying shear wave: a single sine mode keeps its
    shape and its amplitude falls by exp(-nu k^2 t), so the residual over K
    steps is exp(nu k^2 K) - 1 whatever the norm (this fixes the K-step
    offset and which field is the numerator's reference);
  * the solver's residual (one call over T steps) equals the residual of the
    fields of two separate runs of T - K and K steps.
"""
import math

import numpy as np
import pytest


def _hand_field():
    """4 x 3 lattice, cells in row-major order c = y * 4 + x.

    fluid c0:  u = (1, 0),   u_prev = (0, 0)   |du|_1 = 1, |u|_1 = 1
    fluid c1:  u = (0, -2),  u_prev = (0, 1)   |du|_1 = 3, |u|_1 = 2
    fluid c2:  u = (3, 4),   u_prev = (3, 4)   |du|_1 = 0, |u|_1 = 7
    solid c3:  u = (100, 100), u_prev = (0, 0) (not counted)
    every other cell is solid with u = u_prev = 0.

    r = (1 + 3 + 0) / (1 + 2 + 7) = 4 / 10 = 0.4 exactly.
    Plausible mistakes give other values:
      L2 norms:               sqrt(1 + 9) / sqrt(1 + 4 + 25)   = 0.577...
      no absolute values:     (1 - 3) / (1 - 2 + 7)            = -1/3
      solid cells counted:    (4 + 200) / (10 + 200)           = 0.971...
      numerator/denominator:  10 / 4                           = 2.5
    """
    nx, ny = 4, 3
    solid = np.ones((ny, nx), np.uint8)
    ux = np.zeros((ny, nx))
    uy = np.zeros((ny, nx))
    uxp = np.zeros((ny, nx))
    uyp = np.zeros((ny, nx))
    flat = [a.reshape(-1) for a in (ux, uy, uxp, uyp)]
    rows = [(0, 1, 0, 0, 0), (1, 0, -2, 0, 1), (2, 3, 4, 3, 4)]
    for c, a, b, ap, bp in rows:
        solid.reshape(-1)[c] = 0
        flat[0][c], flat[1][c], flat[2][c], flat[3][c] = a, b, ap, bp
    flat[0][3] = flat[1][3] = 100.0
    return nx, ny, solid, ux, uy, uxp, uyp


def test_residual_of_a_hand_worked_field(ora):
    nx, ny, solid, ux, uy, uxp, uyp = _hand_field()
    p = ora.make_params(nx, ny, 0.8)
    r = ora.residual(p, solid, ux, uy, uxp, uyp)
    assert r == 0.4
    # symmetric in which field is "previous" only in the numerator: swapping
    # the two fields changes the denominator to sum |u_prev|_1 = 0 + 1 + 7 = 8
    assert ora.residual(p, solid, uxp, uyp, ux, uy) == 4.0 / 8.0


def test_residual_of_a_decaying_shear_wave(ora):
    """u_x = A(t) sin(2 pi y / N) in a periodic box keeps its shape and decays
    as A(t) = A(0) exp(-nu k^2 t); r over K steps is exp(nu k^2 K) - 1."""
    N, tau, K = 64, 0.8, 100
    cells = np.zeros((N, N), np.uint8)
    p = ora.make_params(N, N, tau, 1.0, 0.0, periodic=True)
    y = np.arange(N)[:, None] * np.ones((1, N))
    mode = np.sin(2 * np.pi * y / N)
    f = ora.init_state(p, cells, np.ones((N, N)), 1e-4 * mode, np.zeros((N, N)))
    f1, _, uxp, uyp, st1 = ora.run(p, cells, np.zeros(N), f, 400)
    _, _, ux, uy, st2 = ora.run(p, cells, np.zeros(N), f1, K)
    assert st1 == 0 and st2 == 0
    r = ora.residual(p, cells, ux, uy, uxp, uyp)
    nu = (tau - 0.5) / 3.0
    k = 2 * np.pi / N
    expected = math.exp(nu * k * k * K) - 1.0
    assert r == pytest.approx(expected, rel=1e-2)
    # an offset of two steps either way (K +- 2) moves the closed form by 2 %
    assert abs(r - (math.exp(nu * k * k * (K + 2)) - 1.0)) > 0.5 * abs(r - expected)


def test_solver_residual_equals_two_separate_runs(ora):
    from paper_1303_0107_gb300 import inputs as I
    cfg = I.config_t_junction()
    cells = cfg["cells"]
    ny, nx = cells.shape
    K, T = 100, 600
    p = ora.make_params(nx, ny, cfg["tau"], 1.0, cfg["u_max"])
    s = ora.Solver(p, cells, residual_every=K)
    r = s.solve(T)["residual"]
    u_in = ora.inlet_profile(p, cells)
    f = ora.init(p, cells)
    f, _, uxp, uyp, _ = ora.run(p, cells, u_in, f, T - K)
    _, _, ux, uy, _ = ora.run(p, cells, u_in, f, K)
    fluid = cells == 0
    num = np.abs(ux - uxp)[fluid].sum() + np.abs(uy - uyp)[fluid].sum()
    den = np.abs(ux)[fluid].sum() + np.abs(uy)[fluid].sum()
    assert r == pytest.approx(num / den, rel=1e-12)
    assert 0 < r < 1
