"""Pins of the oracle's collision models beyond BGK (regularised BGK and the
Smagorinsky eddy-viscosity closure): what the mathematics fixes about them."""
import math

import numpy as np
import pytest

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def _feq(rho, ux, uy):
    cu = CX[:, None, None] * ux + CY[:, None, None] * uy
    return W[:, None, None] * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (ux ** 2 + uy ** 2))


def _random_state(ora, N, seed, amp=0.02):
    rng = np.random.default_rng(seed)
    rho = 1 + amp * rng.standard_normal((N, N))
    ux = amp * rng.standard_normal((N, N))
    uy = amp * rng.standard_normal((N, N))
    f = _feq(rho, ux, uy) * (1 + 0.05 * rng.standard_normal((9, N, N)))  # plus arbitrary non-equilibrium
    return f.astype(np.float64)


def _one_step(ora, f, N, tau, collision, c_smag=0.0):
    p = ora.make_params(N, N, tau, 1.0, 0.0, periodic=True, collision=collision, c_smag=c_smag)
    cells = np.zeros((N, N), np.uint8)
    out, rho, ux, uy, st = ora.run(p, cells, np.zeros(N), f.reshape(9, N * N).copy().reshape(9, N, N), 1)
    assert st == 0
    return out


@pytest.mark.parametrize("collision", [1, 2])
@pytest.mark.parametrize("tau", [0.53, 0.8, 1.2])
def test_shear_wave_viscosity_of_each_model(ora, collision, tau):
    """Both models keep nu = (tau - 1/2)/3 (Sec. 2.1) for a small shear wave:
    the regularisation only removes modes above second order, and the eddy
    viscosity of a wave of amplitude 1e-6 is negligible at c_smag = 0.1."""
    N = 64
    cells = np.zeros((N, N), np.uint8)
    p = ora.make_params(N, N, tau, 1.0, 0.0, periodic=True, collision=collision, c_smag=0.1)
    y = np.arange(N)[:, None] * np.ones((1, N))
    mode = np.sin(2 * np.pi * y / N)
    f = ora.init_state(p, cells, np.ones((N, N)), 1e-6 * mode, np.zeros((N, N)))
    nu = (tau - 0.5) / 3
    k = 2 * np.pi / N
    dt = int(1.0 / (nu * k * k))
    f1, _, ux1, _, _ = ora.run(p, cells, np.zeros(N), f, 200)
    _, _, ux2, _, _ = ora.run(p, cells, np.zeros(N), f1, dt)
    nu_m = math.log((ux1 * mode).sum() / (ux2 * mode).sum()) / (k * k * dt)
    assert nu_m == pytest.approx(nu, rel=0.01)


def test_regularised_equals_bgk_where_the_projection_changes_nothing(ora):
    N = 8
    # at tau = 1 both relax fully to f^eq
    f = _random_state(ora, N, 1)
    a = _one_step(ora, f, N, 1.0, 0)
    b = _one_step(ora, f, N, 1.0, 1)
    assert np.abs(a - b).max() <= 1e-15
    # a uniform state (streaming moves nothing) whose non-equilibrium part is
    # already the second-order Hermite projection: BGK and the regularised
    # collision agree at any tau
    rho, ux, uy, pxx, pyy, pxy = 1.03, 0.02, -0.01, 1e-3, -4e-4, 2e-4
    eq = _feq(np.full((N, N), rho), np.full((N, N), ux), np.full((N, N), uy))
    cs2 = 1 / 3
    q = (CX ** 2 - cs2) * pxx + (CY ** 2 - cs2) * pyy + 2 * CX * CY * pxy
    f = eq + (W * q / (2 * cs2 * cs2))[:, None, None]
    a = _one_step(ora, f, N, 0.7, 0)
    b = _one_step(ora, f, N, 0.7, 1)
    assert np.abs(a - b).max() <= 1e-15


def test_smagorinsky_without_constant_is_bgk(ora):
    N = 8
    f = _random_state(ora, N, 2)
    a = _one_step(ora, f, N, 0.6, 0)
    b = _one_step(ora, f, N, 0.6, 2, c_smag=0.0)
    assert np.abs(a - b).max() <= 1e-15


def test_smagorinsky_relaxation_time_solves_its_quadratic(ora):
    """tau_eff is the positive root of t^2 - tau t - C^2 sqrt(2 Pi:Pi) / (2 rho c_s^4) = 0."""
    L = ora.lib()
    cs4 = 1 / 9
    rng = np.random.default_rng(4)
    prev = None
    for k in range(200):
        tau, c, rho = 0.5 + rng.random(), 0.05 + 0.2 * rng.random(), 0.9 + 0.2 * rng.random()
        pxx, pyy, pxy = 1e-2 * rng.standard_normal(3)
        t = L.ora_smagorinsky_tau(tau, c, rho, pxx, pyy, pxy)
        pp = pxx * pxx + pyy * pyy + 2 * pxy * pxy
        b = c * c * math.sqrt(2 * pp) / (2 * rho * cs4)
        assert abs(t * t - tau * t - b) <= 1e-13 * max(1.0, t * t)
        assert t >= tau
    # more stress, more eddy viscosity
    ts = [L.ora_smagorinsky_tau(0.6, 0.1, 1.0, s, 0.0, 0.0) for s in (0.0, 1e-4, 1e-3, 1e-2)]
    assert ts[0] == pytest.approx(0.6, abs=1e-15) and all(a < b for a, b in zip(ts, ts[1:]))


@pytest.mark.parametrize("collision", [1, 2])
def test_mass_conserved_in_closed_box(ora, collision):
    N = 32
    cells = np.zeros((N, N), np.uint8)
    cells[0, :] = cells[-1, :] = cells[:, 0] = cells[:, -1] = 1
    p = ora.make_params(N, N, 0.55, 1.0, 0.0, periodic=True, collision=collision, c_smag=0.15)
    rng = np.random.default_rng(5)
    fluid = cells == 0
    rho = 1 + 0.01 * rng.standard_normal((N, N)) * fluid
    ux = 0.01 * rng.standard_normal((N, N)) * fluid
    uy = 0.01 * rng.standard_normal((N, N)) * fluid
    f = ora.init_state(p, cells, rho, ux, uy)
    m0 = f[:, fluid].sum()
    f2, *_ = ora.run(p, cells, np.zeros(N), f, 2000)
    assert abs(f2[:, fluid].sum() - m0) <= 1e-12 * m0


def test_smagorinsky_stable_where_bgk_diverges(ora):
    """A channel with a square block at tau = 0.51 and u_max = 0.05 (Re about
    870 on the channel width): BGK blows up within 2000 steps, the eddy
    viscosity keeps the solution bounded (measured on this oracle)."""
    nx, ny = 200, 60
    cells = np.ones((ny, nx), np.uint8)
    cells[1:-1, :] = 0
    cells[22:38, 50:56] = 1
    p = ora.make_params(nx, ny, 0.51, 1.0, 0.05)
    with pytest.raises(FloatingPointError):
        ora.Solver(p, cells, residual_every=0).solve(2000)
    p = ora.make_params(nx, ny, 0.51, 1.0, 0.05, collision=2, c_smag=0.1)
    s = ora.Solver(p, cells, residual_every=0)
    r = s.solve(2000)
    assert np.isfinite(r["dp"]) and np.abs(s.ux).max() < 0.2
