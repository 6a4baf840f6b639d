"""Pins of the D3Q19 oracle against facts that do not come from the oracle:
the moment identities of the lattice, the exact reduction of z-, y- and
x-invariant flows to the (separately pinned) D2Q9 oracle, shear-wave decay at
the viscosity nu = (tau - 1/2)/3, plane and square-duct Poiseuille flow from
their closed-form solutions, and brute-force checks of the outlet regions,
observables and exchange scores."""
import itertools
import math

import numpy as np
import pytest

import oracle as ora2
from oracle import lbm3d as o3

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

WRAP_ALL = 7


def test_lattice_moments_are_isotropic_to_fourth_order():
    cx, cy, cz, opp, w, cs2 = o3.lattice3()
    c = np.stack([cx, cy, cz], 1).astype(float)
    # the 19 velocities are exactly the vectors of {-1,0,1}^3 with |c|^2 <= 2
    want = {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(a * a for a in v) <= 2}
    assert {tuple(int(a) for a in v) for v in c} == want and len(c) == 19
    assert np.array_equal(c[opp], -c)
    assert cs2 == pytest.approx(1 / 3, abs=1e-16)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    d = np.eye(3)
    for a, b in itertools.product(range(3), repeat=2):
        assert (w * c[:, a] * c[:, b]).sum() == pytest.approx(cs2 * d[a, b], abs=1e-15)
        assert abs((w * c[:, a]).sum()) < 1e-16
        for g in range(3):
            assert abs((w * c[:, a] * c[:, b] * c[:, g]).sum()) < 1e-16
            for h in range(3):
                iso = cs2 * cs2 * (d[a, b] * d[g, h] + d[a, g] * d[b, h] + d[a, h] * d[b, g])
                assert (w * c[:, a] * c[:, b] * c[:, g] * c[:, h]).sum() == pytest.approx(iso, abs=1e-15)


def test_equilibrium_moments():
    cx, cy, cz, _, _, cs2 = o3.lattice3()
    c = np.stack([cx, cy, cz], 1).astype(float)
    rng = np.random.default_rng(3)
    for _ in range(5):
        rho = 1 + 0.1 * rng.standard_normal()
        u = 0.05 * rng.standard_normal(3)
        fe = np.array([o3.feq3(i, rho, *u) for i in range(19)])
        assert fe.sum() == pytest.approx(rho, abs=1e-14)
        assert np.allclose(c.T @ fe, rho * u, atol=1e-15)
        pi = np.einsum("i,ia,ib->ab", fe, c, c)
        assert np.allclose(pi, rho * cs2 * np.eye(3) + rho * np.outer(u, u), atol=1e-15)
    # at rest the equilibrium is w rho
    assert [o3.feq3(i, 2.0, 0, 0, 0) for i in range(19)] == pytest.approx(2.0 * o3.lattice3()[4], abs=1e-16)


def test_regularisation_keeps_the_moments_up_to_second_order():
    """The regularisation of the port cells replaces f by f^eq plus the
    second-order Hermite projection of f - f^eq: density, momentum and all
    six components of the momentum flux are kept, the higher non-equilibrium
    moments are removed, and a second application changes nothing."""
    cx, cy, cz, _, w, cs2 = o3.lattice3()
    c = np.stack([cx, cy, cz], 1).astype(float)
    rng = np.random.default_rng(8)
    for _ in range(4):
        f = w * (1 + 0.2 * rng.standard_normal(19))
        rho = f.sum()
        u = c.T @ f / rho
        g = o3.regularize3(f, rho, *u)
        assert g.sum() == pytest.approx(rho, abs=1e-15)
        assert np.allclose(c.T @ g, c.T @ f, atol=1e-15)
        assert np.allclose(np.einsum("i,ia,ib->ab", g, c, c), np.einsum("i,ia,ib->ab", f, c, c), atol=1e-15)
        fe = np.array([o3.feq3(i, rho, *u) for i in range(19)])
        # g - f^eq lies in the span of w_i (c_ia c_ib - c_s^2 delta_ab)
        basis = np.stack([w * (c[:, a] * c[:, b] - cs2 * (a == b))
                          for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))], 1)
        coef = np.linalg.lstsq(basis, g - fe, rcond=None)[0]
        assert np.abs(basis @ coef - (g - fe)).max() < 1e-15
        assert np.allclose(o3.regularize3(g, rho, *u), g, atol=1e-16)
        assert np.abs(g - f).max() > 1e-3          # it did change a generic f


def _obstacles_2d(ny, nx, seed):
    rng = np.random.default_rng(seed)
    s = np.zeros((ny, nx), np.uint8)
    for _ in range(3):
        y, x = rng.integers(0, ny - 3), rng.integers(0, nx - 3)
        s[y:y + rng.integers(1, 4), x:x + rng.integers(1, 4)] = 1
    return s


def _smooth_state(shape, seed):
    ny, nx = shape
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, 4)
    rho = 1 + 0.02 * np.sin(2 * np.pi * xx / nx + ph[0]) * np.cos(2 * np.pi * yy / ny + ph[1])
    ua = 0.04 * np.sin(2 * np.pi * yy / ny + ph[2])
    ub = 0.03 * np.cos(2 * np.pi * xx / nx + ph[3])
    return rho, ua, ub


@pytest.mark.parametrize("axis", ["z", "y", "x"])
def test_invariant_flow_reduces_to_d2q9_oracle(axis):
    """A flow that does not change along one axis and has no velocity along
    it: summing the D3Q19 populations over that axis's component gives D2Q9
    populations (weights 4/9, 1/9, 1/36 and the same second-order equilibrium),
    and the streaming, bounce-back and BGK collision commute with the sum; so
    the 3D oracle must follow the 2D oracle step by step to rounding."""
    cx, cy, cz, _, _, _ = o3.lattice3()
    c2x, c2y, _, _, _ = ora2.lattice()
    n2y, n2x, tau, steps = 14, 18, 0.7, 60
    s2 = _obstacles_2d(n2y, n2x, 5)
    rho2, ua, ub = _smooth_state((n2y, n2x), 6)
    ua, ub = ua * (s2 == 0), ub * (s2 == 0)
    # (a, b) of the 2D plane -> 3D axes; k is the invariant axis
    if axis == "z":
        shape, a_of, b_of, k_c = (3, n2y, n2x), cx, cy, cz          # 2D (x, y) = 3D (x, y)
        s3 = np.broadcast_to(s2, shape)
        vel = lambda: (np.broadcast_to(ua, shape), np.broadcast_to(ub, shape), np.zeros(shape))
        take = lambda a3: a3[0]
    elif axis == "y":
        shape, a_of, b_of, k_c = (n2y, 3, n2x), cx, cz, cy          # 2D (x, y) = 3D (x, z)
        s3 = np.broadcast_to(s2[:, None, :], shape)
        vel = lambda: (np.broadcast_to(ua[:, None, :], shape), np.zeros(shape), np.broadcast_to(ub[:, None, :], shape))
        take = lambda a3: a3[:, 0, :]
    else:
        shape, a_of, b_of, k_c = (n2y, n2x, 4), cy, cz, cx          # 2D (x, y) = 3D (y, z)
        s3 = np.broadcast_to(s2[:, :, None], shape)
        vel = lambda: (np.zeros(shape), np.broadcast_to(ua[:, :, None], shape), np.broadcast_to(ub[:, :, None], shape))
        take = lambda a3: a3[:, :, 0]
    nz, ny, nx = shape
    s3 = np.ascontiguousarray(s3, np.uint8)
    rho3 = np.broadcast_to(rho2 if axis == "z" else (rho2[:, None, :] if axis == "y" else rho2[:, :, None]), shape)
    p3 = o3.make_params3(nx, ny, nz, tau, periodic=WRAP_ALL)
    p2 = ora2.make_params(n2x, n2y, tau, periodic=True)
    f3 = o3.init_state3(p3, s3, rho3, *vel())
    f2 = ora2.init_state(p2, s2, rho2, ua, ub)

    def project(f):
        out = np.zeros((9, n2y, n2x))
        for i in range(19):
            j = int(np.flatnonzero((c2x == a_of[i]) & (c2y == b_of[i]))[0])
            out[j] += take(f[i])
        return out

    assert np.abs(project(f3) - f2).max() < 1e-15
    f3, r3, *_ , st3 = o3.run3(p3, s3, np.zeros((nz, ny)), f3, steps)
    f2, r2, _, _, st2 = ora2.run(p2, s2, np.zeros(n2y), f2, steps)
    assert st3 == 0 and st2 == 0
    # still invariant along the axis, and equal to the 2D run
    for i in range(19):
        assert np.abs(np.moveaxis(f3[i], {"z": 0, "y": 1, "x": 2}[axis], 0) - take(f3[i])).max() == 0.0
    assert np.abs(project(f3) - f2).max() < 1e-13
    assert np.abs(take(r3) - r2).max() < 1e-13
    assert np.abs(f2).max() > 0.01 and np.abs(np.diff(f2, axis=2)).max() > 1e-4  # a real flow


def test_closed_box_conserves_mass_and_momentum():
    shape = (6, 7, 8)
    rng = np.random.default_rng(1)
    solid = np.zeros(shape, np.uint8)
    p = o3.make_params3(8, 7, 6, 0.62, periodic=WRAP_ALL)
    rho = 1 + 0.01 * rng.standard_normal(shape)
    u = [0.02 * rng.standard_normal(shape) for _ in range(3)]
    f0 = o3.init_state3(p, solid, rho, *u)
    f, r, ux, uy, uz, st = o3.run3(p, solid, np.zeros((6, 7)), f0, 50)
    cx, cy, cz, *_ = o3.lattice3()
    assert f.sum() == pytest.approx(f0.sum(), rel=1e-14)
    for cc in (cx, cy, cz):
        j0 = np.tensordot(cc.astype(float), f0, 1).sum()
        j1 = np.tensordot(cc.astype(float), f, 1).sum()
        assert abs(j1 - j0) < 1e-13
    # with walls (an obstacle) mass alone is conserved
    solid[2:4, 2:5, 3:6] = 1
    f0 = o3.init_state3(p, solid, rho, *u)
    f, *_ = o3.run3(p, solid, np.zeros((6, 7)), f0, 50)
    assert f.sum() == pytest.approx(f0.sum(), rel=1e-14)


def _shear_wave_rate_error(n, k, tau):
    """Relative error of the measured decay rate of u_x = A sin(k . r) against
    nu |k|^2, measured over one e-folding after a short settling time."""
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    kv = 2 * np.pi / n * np.array(k, float)
    phase = kv[0] * z + kv[1] * y + kv[2] * x
    solid = np.zeros((n, n, n), np.uint8)
    p = o3.make_params3(n, n, n, tau, periodic=WRAP_ALL)
    nu = (tau - 0.5) / 3
    T = int(1 / (nu * (kv @ kv)))
    f0 = o3.init_state3(p, solid, np.ones_like(phase), 1e-4 * np.sin(phase), np.zeros_like(phase),
                        np.zeros_like(phase))
    f1, _, ux1, *_ = o3.run3(p, solid, np.zeros((n, n)), f0, T // 5)
    _, _, ux2, uy, uz, st = o3.run3(p, solid, np.zeros((n, n)), f1, T)
    a1, a2 = (2 * (u * np.sin(phase)).mean() for u in (ux1, ux2))
    assert np.abs(uy).max() < 1e-12 and np.abs(uz).max() < 1e-12
    return -math.log(a2 / a1) / T / (nu * (kv @ kv)) - 1


@pytest.mark.parametrize("tau", [0.6, 0.8])
def test_shear_wave_decays_at_the_lattice_viscosity(tau):
    """A shear wave in a periodic cube decays as exp(-nu |k|^2 t) with
    nu = (tau - 1/2)/3 (the relation of tau and viscosity of Sec. 2.1), up to
    the scheme's second-order error: halving the wavelength's resolution
    multiplies the error by four."""
    e16, e32 = (_shear_wave_rate_error(n, (1, 0, 0), tau) for n in (16, 32))   # k along z
    assert abs(e32) < 4e-3 and 3.5 < e16 / e32 < 4.5
    assert abs(_shear_wave_rate_error(32, (1, 1, 0), tau)) < 2e-3                # k along z + y


MAGIC_TAU = 0.5 + math.sqrt(3.0 / 16.0)  # BGK + halfway bounce-back: plane Poiseuille exact


def _channel(nx, ny, nz, duct):
    s = np.zeros((nz, ny, nx), np.uint8)
    s[0], s[-1] = 1, 1
    if duct:
        s[:, 0], s[:, -1] = 1, 1
    return s


def test_plane_poiseuille_between_z_walls():
    """Walls at z = 1/2 and z = H + 1/2, y wrapped: the developed profile is
    the parabola u(z) = 6 U s (1 - s), s = (z - 1/2)/H, with the mean speed U
    set by the pressure gradient, U = G H^2 / (12 mu), p = rho/3."""
    nx, ny, H, tau, umax = 64, 3, 10, MAGIC_TAU, 2e-3
    s = _channel(nx, ny, H + 2, duct=False)
    p = o3.make_params3(nx, ny, H + 2, tau, u_max=umax, periodic=2)
    sv = o3.Solver3(p, s)
    out = sv.solve(4000)
    z = np.arange(1, H + 1)
    sz = (z - 0.5) / H
    mid = slice(24, 40)
    prof = sv.ux[1:H + 1, 1, mid].mean(axis=1)
    q = sz * (1 - sz)
    amp = (prof @ q) / (q @ q)                  # least-squares parabola through the cell centres
    assert np.abs(prof - amp * q).max() < 1e-5 * prof.max()   # exact at this tau
    U = amp / 6                                 # mean speed of the continuous parabola
    # the inlet imposes exactly the parabola of the 2D method, the outlet rho0
    assert np.array_equal(sv.u_in[:, 1] > 0, s[:, 1, 0] == 0)
    assert np.abs(sv.ux[1:H + 1, :, 0] - sv.u_in[1:H + 1, :]).max() < 1e-15
    assert np.abs(sv.rho[1:H + 1, :, -1] - 1.0).max() < 1e-15
    rho_line = sv.rho[1:H + 1, 1, :].mean(axis=0)
    G = -np.polyfit(np.arange(24, 40), rho_line[mid] / 3, 1)[0]
    mu = (tau - 0.5) / 3
    assert U == pytest.approx(G * H * H / (12 * mu), rel=5e-3)
    assert out["m_out"].sum() == pytest.approx(out["m_in"], rel=5e-4)
    assert len(out["m_out"]) == 1


def _duct_series(a, y, z, terms=60):
    """Square duct |y|, |z| < a, -dp/dx = G: u(y, z) mu / (G a^2)."""
    s = 0.0
    for n in range(1, 2 * terms, 2):
        b = n * np.pi / (2 * a)
        s = s + (-1) ** ((n - 1) // 2) / n ** 3 * (1 - np.cosh(b * z) / np.cosh(b * a)) * np.cos(b * y)
    return 16 * a * a / np.pi ** 3 * s / (a * a)


def test_square_duct_poiseuille():
    """Developed flow in a square duct against its Fourier-series solution:
    the shape of the cross-section profile and the centre speed per unit
    pressure gradient."""
    nx, W, tau, umax = 56, 10, MAGIC_TAU, 2e-3
    s = _channel(nx, W + 2, W + 2, duct=True)
    p = o3.make_params3(nx, W + 2, W + 2, tau, u_max=umax)
    sv = o3.Solver3(p, s)
    out = sv.solve(4000)
    a = W / 2
    c = np.arange(1, W + 1) - 0.5 - a                         # cell centres, walls at +-a
    zz, yy = np.meshgrid(c, c, indexing="ij")
    shape = _duct_series(a, yy, zz)
    mid = slice(22, 34)
    prof = sv.ux[1:W + 1, 1:W + 1, mid].mean(axis=2)
    assert np.abs(prof / prof.max() - shape / shape.max()).max() < 5e-3
    rho_line = sv.rho[1:W + 1, 1:W + 1, :].mean(axis=(0, 1))
    G = -np.polyfit(np.arange(22, 34), rho_line[mid] / 3, 1)[0]
    mu = (tau - 0.5) / 3
    centre = prof[W // 2 - 1:W // 2 + 1, W // 2 - 1:W // 2 + 1].mean()
    want = (G * a * a / mu) * _duct_series(a, np.array([0.5, -0.5]), np.array([0.5, -0.5])).mean()
    assert centre == pytest.approx(want, rel=1e-2)
    assert out["m_out"].sum() == pytest.approx(out["m_in"], rel=5e-4)
    # symmetric under exchanging y and z
    assert np.abs(prof - prof.T).max() < 1e-12 * prof.max()


def test_outlet_regions_match_connected_components():
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(9)
    nz, ny, nx = 9, 11, 6
    s = np.ones((nz, ny, nx), np.uint8)
    face = rng.random((nz - 2, ny - 2)) < 0.5
    s[1:-1, 1:-1, -1] = ~face
    s[1:-1, 1:-1, -2] = 0
    p = o3.make_params3(nx, ny, nz, 0.8)
    ids, n = o3.outlet_ids3(p, s)
    lab, m = ndi.label(s[:, :, -1] == 0)        # 4-connectivity, numbered in raster order
    assert n == m
    assert np.array_equal(ids, lab - 1)


def test_observables_by_brute_force():
    rng = np.random.default_rng(4)
    nz, ny, nx = 7, 8, 9
    s = np.ones((nz, ny, nx), np.uint8)
    s[1:-1, 1:-1, :] = (rng.random((nz - 2, ny - 2, nx)) < 0.2).astype(np.uint8)
    s[1:-1, 1:-1, 0:2] = 0
    s[1:-1, 1:-1, -2:] = 0
    s[3, 1:-1, -1] = 1                           # splits the outlet face in two
    p = o3.make_params3(nx, ny, nz, 0.8)
    ids, n = o3.outlet_ids3(p, s)
    rho = 1 + 0.1 * rng.random(s.shape)
    ux = 0.1 * rng.standard_normal(s.shape)
    dp, m_in, m_out = o3.observables3(p, s, rho, ux, ids, n)
    fi, fo = s[:, :, 0] == 0, s[:, :, -1] == 0
    want = rho[:, :, 0][fi].mean() / 3 - rho[:, :, -1][fo].mean() / 3
    assert dp == pytest.approx(want, rel=1e-13)
    assert m_in == pytest.approx((rho * ux)[:, :, 0][fi].sum(), rel=1e-13)
    assert n == 2
    for r in range(n):
        sel = ids == r
        assert m_out[r] == pytest.approx((rho * ux)[:, :, -1][sel].sum(), rel=1e-13)


@pytest.mark.parametrize("axis", ["z", "y"])
def test_scores_of_an_extruded_layer_equal_the_2d_scores(axis):
    """In a geometry extruded along z (or y) with no velocity along it, the
    cells of an inner layer see solid/fluid neighbours along that axis of
    their own kind, so candidates and scores (Eqs. 5-6) are those of the 2D
    oracle on the layer's plane."""
    rng = np.random.default_rng(2)
    n2y, n2x, tau = 12, 16, 0.7
    s2 = np.ones((n2y, n2x), np.uint8)
    s2[1:-1, :] = (rng.random((n2y - 2, n2x)) < 0.35).astype(np.uint8)
    rho2 = 1 + 0.05 * rng.random((n2y, n2x))
    ua, ub = 0.05 * rng.standard_normal((2, n2y, n2x))
    p2 = ora2.make_params(n2x, n2y, tau)
    c2, sc2 = ora2.scores(p2, s2, rho2, ua, ub)
    depth = 5
    if axis == "z":
        shape = (depth, n2y, n2x)
        ex = lambda a: np.ascontiguousarray(np.broadcast_to(a, shape))
        vel = (ex(ua), ex(ub), np.zeros(shape))
        take = lambda a: a[2]
    else:
        shape = (n2y, depth, n2x)
        ex = lambda a: np.ascontiguousarray(np.broadcast_to(a[:, None, :], shape))
        vel = (ex(ua), np.zeros(shape), ex(ub))
        take = lambda a: a[:, 2, :]
    nz, ny, nx = shape
    p3 = o3.make_params3(nx, ny, nz, tau)
    c3, sc3 = o3.scores3(p3, ex(s2).astype(np.uint8), ex(rho2), *vel)
    assert np.array_equal(take(c3), c2) and c2.any()
    assert np.allclose(take(sc3), sc2, rtol=1e-14, atol=0)


def test_exchange_keeps_the_volume_and_resets_the_swapped_cells():
    nx, W, tau = 24, 8, 0.8
    s = _channel(nx, W + 2, W + 2, duct=True)
    s[3:7, 3:7, 10:14] = 1
    p = o3.make_params3(nx, W + 2, W + 2, tau, u_max=0.01)
    sv = o3.Solver3(p, s)
    sv.solve(200)
    before = int((sv.solid == 0).sum())
    fi, si = sv.pick(5)
    assert len(fi) == len(si) == 5
    flat = sv.solid.reshape(-1)
    assert np.all(flat[fi] == 0) and np.all(flat[si] == 1)
    out = sv.optimize_step(5, 100)
    assert out["fluid_count"] == before and int((sv.solid == 0).sum()) == before
    assert np.all(sv.solid.reshape(-1)[out["solid_idx"]] == 0)
    assert np.all(sv.solid.reshape(-1)[out["fluid_idx"]] == 1)


def _random_cell(rng, scale=0.1):
    cx, cy, cz, _, w, _ = o3.lattice3()
    return w * (1 + scale * rng.standard_normal(19))


def _moments(f):
    cx, cy, cz, _, _, _ = o3.lattice3()
    c = np.stack([cx, cy, cz], 1).astype(float)
    rho = f.sum()
    return rho, c.T @ f / rho, c


@pytest.mark.parametrize("collision,c_smag", [(o3.COLLIDE_BGK, 0.0), (o3.COLLIDE_REGULARIZED, 0.0),
                                              (o3.COLLIDE_SMAGORINSKY, 0.0), (o3.COLLIDE_SMAGORINSKY, 0.3)])
def test_collision_models_relax_the_stress_as_defined(collision, c_smag):
    """One cell: every model keeps rho and j; BGK scales f - f^eq by
    (1 - 1/tau); the regularised model scales the six components of the
    non-equilibrium stress by (1 - 1/tau) and leaves f - f^eq in the
    second-order Hermite span; the Smagorinsky model is BGK at tau_eff, where
    tau_eff - tau = nu_t / c_s^2 with nu_t = C^2 |S|, |S| = sqrt(2 S:S) and
    S = -Pi / (2 rho c_s^2 tau_eff) (the closure's definition)."""
    cx, cy, cz, _, w, cs2 = o3.lattice3()
    tau = 0.7
    p = o3.make_params3(4, 3, 3, tau, collision=collision, c_smag=c_smag)
    rng = np.random.default_rng(21)
    for _ in range(4):
        f = _random_cell(rng)
        rho, u, c = _moments(f)
        fe = np.array([o3.feq3(i, rho, *u) for i in range(19)])
        g, tau_eff = o3.collide3(p, f)
        assert g.sum() == pytest.approx(rho, abs=1e-15) and np.allclose(c.T @ g, c.T @ f, atol=1e-15)
        pi0 = np.einsum("i,ia,ib->ab", f - fe, c, c)
        pi1 = np.einsum("i,ia,ib->ab", g - fe, c, c)
        if collision == o3.COLLIDE_REGULARIZED:
            assert np.allclose(pi1, (1 - 1 / tau) * pi0, atol=1e-16)
            basis = np.stack([w * (c[:, a] * c[:, b] - cs2 * (a == b))
                              for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))], 1)
            coef = np.linalg.lstsq(basis, g - fe, rcond=None)[0]
            assert np.abs(basis @ coef - (g - fe)).max() < 1e-16
        else:
            if collision == o3.COLLIDE_SMAGORINSKY:
                S = -pi0 / (2 * rho * cs2 * tau_eff)
                nu_t = c_smag ** 2 * np.sqrt(2 * (S * S).sum())
                assert (tau_eff - tau) * cs2 == pytest.approx(nu_t, rel=1e-12, abs=1e-18)
                assert (tau_eff > tau) == (c_smag > 0)
            else:
                assert tau_eff == tau
            assert np.allclose(g - fe, (1 - 1 / tau_eff) * (f - fe), atol=1e-16)
    if collision == o3.COLLIDE_SMAGORINSKY and c_smag == 0.0:  # C = 0 is BGK to the bit
        f = _random_cell(rng)
        assert np.array_equal(o3.collide3(p, f)[0], o3.collide3(o3.make_params3(4, 3, 3, tau), f)[0])


def test_regularised_shear_wave_decays_at_the_lattice_viscosity():
    """The regularised model keeps the viscosity of BGK, nu = (tau - 1/2)/3:
    its shear-wave decay converges to nu |k|^2 at second order."""
    def rate_error(n, tau=0.8):
        z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        k = 2 * np.pi / n
        phase = k * z
        solid = np.zeros((n, n, n), np.uint8)
        p = o3.make_params3(n, n, n, tau, periodic=WRAP_ALL, collision=o3.COLLIDE_REGULARIZED)
        nu = (tau - 0.5) / 3
        T = int(1 / (nu * k * k))
        f0 = o3.init_state3(p, solid, np.ones_like(phase), 1e-4 * np.sin(phase), np.zeros_like(phase),
                            np.zeros_like(phase))
        f1, _, u1, *_ = o3.run3(p, solid, np.zeros((n, n)), f0, T // 5)
        _, _, u2, *_ = o3.run3(p, solid, np.zeros((n, n)), f1, T)
        a1, a2 = (2 * (u * np.sin(phase)).mean() for u in (u1, u2))
        return -math.log(a2 / a1) / T / (nu * k * k) - 1
    e16, e32 = rate_error(16), rate_error(32)
    assert abs(e32) < 4e-3 and 3.3 < e16 / e32 < 4.7


def test_smagorinsky_damps_a_shear_wave_more_as_c_grows_and_c0_is_bgk():
    """The eddy viscosity is non-negative and grows with C: a shear wave of
    finite amplitude ends weaker for every larger C; C = 0 is BGK exactly."""
    n, tau = 16, 0.55
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    phase = 2 * np.pi / n * z
    solid = np.zeros((n, n, n), np.uint8)

    def run(coll, c):
        p = o3.make_params3(n, n, n, tau, periodic=WRAP_ALL, collision=coll, c_smag=c)
        f0 = o3.init_state3(p, solid, np.ones_like(phase), 0.05 * np.sin(phase), np.zeros_like(phase),
                            np.zeros_like(phase))
        f, _, ux, *_ = o3.run3(p, solid, np.zeros((n, n)), f0, 200)
        return f, 2 * (ux * np.sin(phase)).mean()

    f_bgk, a_bgk = run(o3.COLLIDE_BGK, 0.0)
    f_c0, a_c0 = run(o3.COLLIDE_SMAGORINSKY, 0.0)
    assert np.array_equal(f_bgk, f_c0)
    amps = [run(o3.COLLIDE_SMAGORINSKY, c)[1] for c in (0.1, 0.2, 0.5, 1.0)]
    assert a_bgk > amps[0] > amps[1] > amps[2] > amps[3] > 0


def _half_and_whole():
    """A half domain against a plane below its row 0 (the upper half of the
    small 3D tree) and the whole symmetric domain it stands for."""
    from paper_1303_0107_gb300 import inputs as I
    cfg = I.config_tree3d_small()
    half = np.ascontiguousarray(cfg["cells"][:, 17:, :])
    whole = np.ascontiguousarray(np.concatenate([half[:, ::-1, :], half], axis=1))
    return cfg, half, whole


def test_mirror_half_domain_equals_upper_half_of_whole_domain():
    """Sec. 3.3 computes half of a symmetric domain: with the plane below row
    0, the half must follow the upper half of the whole domain (fields, the
    inlet profile, dp; u_y odd across the plane), up to rounding order."""
    cfg, half, whole = _half_and_whole()
    nz, nyh, nx = half.shape
    ph = o3.make_params3(nx, nyh, nz, cfg["tau"], u_max=cfg["u_max"], mirror=True)
    pw = o3.make_params3(nx, 2 * nyh, nz, cfg["tau"], u_max=cfg["u_max"])
    assert o3.check_geometry3(ph, half) == 0 and o3.check_geometry3(pw, whole) == 0
    assert o3.check_geometry3(o3.make_params3(nx, nyh, nz, cfg["tau"]), half) != 0  # row 0 fluid needs the plane
    sh, sw = o3.Solver3(ph, half), o3.Solver3(pw, whole)
    assert np.array_equal(sh.u_in, sw.u_in[:, nyh:])
    oh, ow = sh.solve(300), sw.solve(300)
    up = slice(nyh, 2 * nyh)
    scale = np.abs(sw.ux).max()
    for a, b in ((sh.ux, sw.ux[:, up]), (sh.uy, sw.uy[:, up]), (sh.uz, sw.uz[:, up]), (sh.rho, sw.rho[:, up])):
        assert np.abs(a - b).max() <= 1e-12 * max(scale, 1.0)
    assert np.abs(sw.uy[:, :nyh][:, ::-1] + sw.uy[:, up]).max() <= 1e-12 * scale  # odd across the plane
    assert oh["dp"] == pytest.approx(ow["dp"], rel=1e-12)
    assert oh["m_in"] == pytest.approx(ow["m_in"] / 2, rel=1e-12)
    assert abs(sum(oh["m_out"]) - sum(ow["m_out"]) / 2) <= 1e-12 * abs(sum(ow["m_out"]))


def test_mirror_quarter_domain_equals_a_quarter_of_the_whole_domain():
    """Two planes (below y = 0 and below z = 0): the quarter follows the
    corner block of the whole domain mirrored in both, including the edge
    where both planes meet (both velocity components odd across their
    planes)."""
    from paper_1303_0107_gb300 import inputs as I
    cfg = I.config_tree3d_small()
    q = np.ascontiguousarray(cfg["cells"][17:, 17:, :])
    half = np.concatenate([q[:, ::-1, :], q], axis=1)
    whole = np.ascontiguousarray(np.concatenate([half[::-1], half], axis=0))
    nzq, nyq, nx = q.shape
    pq = o3.make_params3(nx, nyq, nzq, cfg["tau"], u_max=cfg["u_max"], mirror=3)
    pw = o3.make_params3(nx, 2 * nyq, 2 * nzq, cfg["tau"], u_max=cfg["u_max"])
    assert o3.check_geometry3(pq, q) == 0 and o3.check_geometry3(pw, whole) == 0
    assert o3.check_geometry3(o3.make_params3(nx, nyq, nzq, cfg["tau"], mirror=1), q) != 0  # z = 0 fluid
    sq, sw = o3.Solver3(pq, q), o3.Solver3(pw, whole)
    assert np.array_equal(sq.u_in, sw.u_in[nzq:, nyq:])
    oq, ow = sq.solve(300), sw.solve(300)
    corner = (slice(nzq, None), slice(nyq, None))
    scale = np.abs(sw.ux).max()
    for a, b in ((sq.ux, sw.ux[corner]), (sq.uy, sw.uy[corner]), (sq.uz, sw.uz[corner]), (sq.rho, sw.rho[corner])):
        assert np.abs(a - b).max() <= 1e-12 * max(scale, 1.0)
    assert np.abs(sw.uz[:nzq][::-1] + sw.uz[nzq:]).max() <= 1e-12 * scale  # u_z odd across the z plane
    assert oq["dp"] == pytest.approx(ow["dp"], rel=1e-12)
    assert oq["m_in"] == pytest.approx(ow["m_in"] / 4, rel=1e-12)
