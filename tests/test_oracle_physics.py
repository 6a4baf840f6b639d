"""Physics pins of the oracle's solver (Sec. 2.1 Eq. 1-4, Sec. 3.3 boundary rules).

Each check is fixed by the mathematics, not by the oracle itself:
  * exact mass conservation of BGK + bounce-back in a closed box;
  * the viscosity of Sec. 2.1, nu = (tau - 1/2)/3, from the decay of a shear wave;
  * plane Poiseuille flow: the parabolic profile and the pressure gradient
    dp/dx = -12 mu U / H^2 of the incompressible limit (Eq. 3), with second-order
    convergence of the profile error in H;
  * the port rules put the imposed moments on the port cells;
  * mirror symmetry of the flow in a mirror-symmetric tree.
"""
import math

import numpy as np
import pytest

from paper_1303_0107_gb300 import inputs as I


def _poiseuille(ora, H, nx, tau, u_max, steps, rule=0, scheme=0):
    cells = I.channel(nx, H)
    p = ora.make_params(nx, H + 2, tau, 1.0, u_max, rule, port_scheme=scheme)
    u_in = ora.inlet_profile(p, cells)
    f = ora.init(p, cells)
    f, rho, ux, uy, st = ora.run(p, cells, u_in, f, steps)
    assert st == 0
    return p, cells, f, rho, ux, uy


def test_closed_box_conserves_mass(ora):
    nx, ny = 64, 32
    cells = I.box(nx, ny)
    p = ora.make_params(nx, ny, 0.7, 1.0, 0.0)
    rng = np.random.default_rng(1)
    rho = 1 + 0.01 * rng.standard_normal((ny, nx))
    ux = 0.01 * rng.standard_normal((ny, nx))
    uy = 0.01 * rng.standard_normal((ny, nx))
    f = ora.init_state(p, cells, rho, ux, uy)
    m0 = f.sum()
    f2, *_ = ora.run(p, cells, np.zeros(ny), f, 10000)
    assert abs(f2.sum() - m0) <= 1e-12 * m0


@pytest.mark.parametrize("tau", [0.53, 0.8, 1.2])
def test_shear_wave_decay_gives_viscosity(ora, tau):
    N = 64
    cells = np.zeros((N, N), np.uint8)
    p = ora.make_params(N, N, tau, 1.0, 0.0, periodic=True)
    y = np.arange(N)[:, None] * np.ones((1, N))
    mode = np.sin(2 * np.pi * y / N)
    f = ora.init_state(p, cells, np.ones((N, N)), 1e-3 * mode, np.zeros((N, N)))
    nu = (tau - 0.5) / 3
    k = 2 * np.pi / N
    t1 = 200
    dt = int(1.0 / (nu * k * k))
    f1, _, ux1, _, _ = ora.run(p, cells, np.zeros(N), f, t1)
    _, _, ux2, _, _ = ora.run(p, cells, np.zeros(N), f1, dt)
    a1 = (ux1 * mode).sum()
    a2 = (ux2 * mode).sum()
    nu_measured = math.log(a1 / a2) / (k * k * dt)
    assert nu_measured == pytest.approx(nu, rel=0.01)


def test_poiseuille_profile_and_pressure_gradient(ora):
    H, nx, tau, u_max = 32, 128, 0.8, 0.01
    p, cells, f, rho, ux, uy = _poiseuille(ora, H, nx, tau, u_max, 30000)
    mid = nx // 2
    s = (np.arange(H) + 0.5) / H
    ana = 4 * u_max * s * (1 - s)
    assert np.abs(ux[1:H + 1, mid] - ana).max() <= 0.01 * u_max
    nu = (tau - 0.5) / 3
    p_line = rho[1:H + 1, :].mean(axis=0) / 3.0
    xs = np.arange(nx // 4, 3 * nx // 4)
    grad = np.polyfit(xs, p_line[xs], 1)[0]
    U = ux[1:H + 1, mid].mean()
    mu = rho[1:H + 1, mid].mean() * nu
    assert grad == pytest.approx(-12 * mu * U / H ** 2, rel=0.01)
    # the reduction of the pressure drop over the whole channel (inlet to outlet
    # cell centres, nx-1 lattice spacings) against the same closed form
    dp, m_in, m_out = ora.observables(p, cells, rho, ux)
    assert dp == pytest.approx(12 * mu * U * (nx - 1) / H ** 2, rel=0.01)


@pytest.mark.slow
def test_poiseuille_second_order_convergence(ora):
    # Zou-He inlet: the profile is imposed on the inlet cells themselves, so the
    # mid-channel error is the bulk scheme's and the walls' alone
    errs = []
    for H, steps in [(8, 4000), (16, 10000), (32, 30000)]:
        p, cells, f, rho, ux, uy = _poiseuille(ora, H, 128, 0.8, 0.01, steps, scheme=ora.PORTS_ZOU_HE)
        s = (np.arange(H) + 0.5) / H
        errs.append(np.abs(ux[1:H + 1, 64] - 0.04 * s * (1 - s)).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.7 < o < 2.3 for o in orders), orders


@pytest.mark.parametrize("scheme", [0, 1])
def test_port_rules_impose_their_moments(ora, scheme):
    H, nx = 16, 64
    p, cells, f, rho, ux, uy = _poiseuille(ora, H, nx, 0.8, 0.02, 500, scheme=scheme)
    u_in = ora.inlet_profile(p, cells)
    fl = slice(1, H + 1)
    # inlet: the rebuilt populations carry exactly u = (u_in(y), 0)
    assert np.abs(ux[fl, 0] - u_in[fl]).max() <= 1e-15
    assert np.abs(uy[fl, 0]).max() <= 1e-16
    # constant-density outlet: rho = rho0, u_y = 0
    assert np.abs(rho[fl, -1] - 1.0).max() <= 1e-15
    assert np.abs(uy[fl, -1]).max() <= 1e-16
    # reported moments are those of the last collision: BGK conserves them
    n = nx * (H + 2)
    ff = f.reshape(9, n)
    cx, cy, *_ = ora.lattice()
    fluid = cells.reshape(-1) == 0
    assert np.abs(ff.sum(axis=0)[fluid] - rho.reshape(-1)[fluid]).max() <= 1e-14
    jx = (cx[:, None] * ff).sum(axis=0)
    assert np.abs(jx[fluid] - (rho * ux).reshape(-1)[fluid]).max() <= 1e-15


def test_regularized_inlet_keeps_the_nonequilibrium_stress(ora):
    """Regularised port: the inlet cell's populations are rebuilt as
    f^eq + w_i/(2 c_s^4) Q_i : Pi, Pi the non-equilibrium stress of the
    populations streamed in with the unknown ones taken by non-equilibrium
    bounce-back.  After the BGK collision the stored populations must therefore
    be f^eq + (1 - 1/tau) * 4.5 w_i Q_i : Pi, with Pi rebuilt here by hand."""
    H, nx, tau = 10, 32, 0.7
    cells = I.channel(nx, H)
    p = ora.make_params(nx, H + 2, tau, 1.0, 0.03)
    u_in = ora.inlet_profile(p, cells)
    f1, *_ = ora.run(p, cells, u_in, ora.init(p, cells), 40)
    f2, (rho, ux, uy) = ora.step_columns(p, cells, u_in, f1, 0, nx)
    cx, cy, opp, w, cs2 = ora.lattice()
    for y in (1, 4, H):  # wall-adjacent and interior inlet cells
        fin = np.zeros(9)
        for i in range(9):
            sx, sy = 0 - cx[i], y - cy[i]
            if sx < 0:
                continue
            fin[i] = f1[opp[i], y, 0] if cells[sy, sx] else f1[i, sy, sx]
        u = u_in[y]
        r = (fin[0] + fin[2] + fin[4] + 2 * (fin[3] + fin[6] + fin[7])) / (1 - u)
        feq = np.array([ora.feq(i, r, u, 0.0) for i in range(9)])
        for i in (1, 5, 8):
            fin[i] = feq[i] + fin[opp[i]] - feq[opp[i]]
        fneq = fin - feq
        pxx, pyy, pxy = (cx * cx * fneq).sum(), (cy * cy * fneq).sum(), (cx * cy * fneq).sum()
        q = (cx * cx - 1 / 3) * pxx + (cy * cy - 1 / 3) * pyy + 2 * cx * cy * pxy
        expect = feq + (1 - 1 / tau) * 4.5 * w * q
        assert rho[y, 0] == pytest.approx(r, rel=1e-14) and ux[y, 0] == pytest.approx(u, rel=1e-13)
        assert np.abs(f2[:, y, 0] - expect).max() <= 1e-15


def test_regularized_ports_stable_where_zou_he_is_not(ora):
    """Reason for the default port scheme: at tau = 0.53 (nu = 0.01) a 64-wide
    channel with a parabolic inlet diverges within a few hundred steps with
    plain Zou-He ports and stays bounded with regularised ones."""
    cells = I.channel(256, 64)
    out = {}
    for scheme in (ora.PORTS_REGULARIZED, ora.PORTS_ZOU_HE):
        p = ora.make_params(256, 66, 0.53, 1.0, 0.0117, port_scheme=scheme)
        f, rho, ux, uy, st = ora.run(p, cells, ora.inlet_profile(p, cells), ora.init(p, cells), 1200)
        m = np.abs(rho - 1)[cells == 0].max()
        out[scheme] = m if np.isfinite(m) else np.inf
    assert out[ora.PORTS_REGULARIZED] < 0.05
    assert out[ora.PORTS_ZOU_HE] > 1.0


def test_inlet_profile_is_parabola_at_cell_centres(ora):
    cells = I.channel(16, 10)
    p = ora.make_params(16, 12, 0.8, 1.0, 0.05)
    u = ora.inlet_profile(p, cells)
    s = (np.arange(10) + 0.5) / 10
    assert np.array_equal(u[0], 0.0) and u[-1] == 0.0
    assert np.allclose(u[1:11], 4 * 0.05 * s * (1 - s), rtol=0, atol=1e-17)
    # two separate inlet runs get a parabola each
    cells2 = cells.copy()
    cells2[5, :] = 1
    p2 = ora.make_params(16, 12, 0.8, 1.0, 0.05)
    u2 = ora.inlet_profile(p2, cells2)
    s4 = (np.arange(4) + 0.5) / 4
    assert np.allclose(u2[1:5], 0.2 * s4 * (1 - s4), atol=1e-17)
    assert u2[5] == 0.0


def test_steady_flux_constant_along_channel(ora):
    """At steady state the flux sum(rho u_x) over a column is the same on every
    column but the last two (the constant-density outlet column pair carries a
    local O(1e-3) disturbance of the reconstruction), and equals the inlet flux."""
    H, nx = 16, 64
    p, cells, f, rho, ux, uy = _poiseuille(ora, H, nx, 1.0, 0.01, 40000, scheme=ora.PORTS_ZOU_HE)
    m = (rho * ux).sum(axis=0)
    interior = m[:nx - 2]
    assert np.abs(interior - m[0]).max() <= 1e-4 * m[0]
    dp, m_in, m_out = ora.observables(p, cells, rho, ux)
    assert m_in == pytest.approx(m[0], rel=1e-15)
    assert m_out.sum() == pytest.approx(m_in, rel=2e-3)


def test_mirror_symmetric_tree_gives_mirror_flow(ora):
    cells = I.tree(128, 64, 2, 8, widths=[8, 4, 4], jitter=0)
    assert np.array_equal(cells, cells[::-1])
    p = ora.make_params(128, 64, 0.8, 1.0, 0.02)
    s = ora.Solver(p, cells)
    r = s.solve(3000)
    m = r["m_out"]
    assert len(m) == 4
    assert np.abs(m - m[::-1]).max() <= 1e-12 * np.abs(m).max()
    assert np.abs(s.ux - s.ux[::-1]).max() <= 1e-13
    assert np.abs(s.uy + s.uy[::-1]).max() <= 1e-13


def test_mirrored_geometry_same_pressure_drop(ora):
    cells = I.tree(128, 64, 2, 8, widths=[8, 4, 4], jitter=2, seed=3)
    p = ora.make_params(128, 64, 0.8, 1.0, 0.02)
    r1 = ora.Solver(p, cells).solve(2000)
    r2 = ora.Solver(p, np.ascontiguousarray(cells[::-1])).solve(2000)
    assert r1["dp"] == pytest.approx(r2["dp"], rel=1e-12)
    assert np.abs(r1["m_out"] - r2["m_out"][::-1]).max() <= 1e-12 * np.abs(r1["m_out"]).max()


def test_neumann_outlet_is_zero_gradient(ora):
    """The zero-gradient outlet of Sec. 3.3: the unknown populations of the
    outlet cell equal the streamed ones of its upstream neighbour, so after one
    step the outlet cell's left-moving populations match those of (nx-2, y)
    pulled from the same state."""
    H, nx = 8, 32
    cells = I.channel(nx, H)
    p = ora.make_params(nx, H + 2, 0.8, 1.0, 0.03, ora.OUT_NEUMANN, port_scheme=ora.PORTS_ZOU_HE)
    u_in = ora.inlet_profile(p, cells)
    f0 = ora.init(p, cells)
    f1, *_ = ora.run(p, cells, u_in, f0, 50)
    # one more step by hand for the outlet column only, from f1
    cx, cy, opp, w, _ = ora.lattice()
    f2, fields = ora.step_columns(p, cells, u_in, f1, 0, nx)
    rho, ux, uy = fields
    for y in range(1, H + 1):
        pulled = {}
        for i in (3, 6, 7):
            sx, sy = nx - 2 - cx[i], y - cy[i]
            pulled[i] = f1[opp[i], y, nx - 2] if cells[sy, sx] else f1[i, sy, sx]
        # rebuild the outlet cell's incoming set and compare its moments
        fin = np.zeros(9)
        for i in range(9):
            sx, sy = nx - 1 - cx[i], y - cy[i]
            if i in (3, 6, 7):
                fin[i] = pulled[i]
            elif cells[sy, sx]:
                fin[i] = f1[opp[i], y, nx - 1]
            else:
                fin[i] = f1[i, sy, sx]
        assert rho[y, nx - 1] == pytest.approx(fin.sum(), rel=1e-14)
        assert ux[y, nx - 1] * rho[y, nx - 1] == pytest.approx((cx * fin).sum(), rel=1e-12, abs=1e-16)
