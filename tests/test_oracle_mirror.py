"""The symmetry plane of Sec. 3.3 (half of the domain computed): a half
domain with the mirror rule below row 0 must reproduce the upper half of the
whole symmetric domain -- fields, populations (reflected) and reductions."""
import numpy as np
import pytest

from paper_1303_0107_gb300 import inputs as I

MIR = [0, 1, 4, 3, 2, 8, 7, 6, 5]


def _symmetric_tree(nx, ny, G, w0):
    full = I.tree(nx, ny, G, w0, ratio=0.5, jitter=0, seed=0)
    assert np.array_equal(full, full[::-1]), "generator output not mirror-symmetric"
    return full


@pytest.mark.parametrize("outlet", [0, 1])
@pytest.mark.parametrize("ports", [0, 1])
def test_half_domain_with_mirror_equals_whole_domain(ora, outlet, ports):
    nx, ny, steps = 160, 64, 600
    full = _symmetric_tree(nx, ny, 2, 16)
    half = full[ny // 2:, :].copy()
    pf = ora.make_params(nx, ny, 0.7, 1.0, 0.04, outlet_rule=outlet, port_scheme=ports)
    ph = ora.make_params(nx, ny // 2, 0.7, 1.0, 0.04, outlet_rule=outlet, port_scheme=ports, mirror=True)
    assert np.array_equal(ora.inlet_profile(ph, half), ora.inlet_profile(pf, full)[ny // 2:])
    sf = ora.Solver(pf, full, residual_every=0)
    sh = ora.Solver(ph, half, residual_every=0)
    of, oh = sf.solve(steps), sh.solve(steps)
    up = slice(ny // 2, ny)
    scale = np.abs(sf.ux).max()
    assert np.abs(sh.ux - sf.ux[up]).max() <= 1e-12 * scale
    assert np.abs(sh.uy - sf.uy[up]).max() <= 1e-12 * scale
    assert np.abs(sh.rho - sf.rho[up]).max() <= 1e-12
    # the lower half of the whole domain is the reflection of the half domain
    low = slice(ny // 2 - 1, None, -1)
    assert np.abs(sf.f[MIR][:, low] - sh.f).max() <= 1e-12
    assert of["dp"] == pytest.approx(oh["dp"], rel=1e-12, abs=1e-15)
    n = len(oh["m_out"])
    assert len(of["m_out"]) == 2 * n
    np.testing.assert_allclose(of["m_out"][n:], oh["m_out"], rtol=1e-11, atol=1e-16)


def test_mirror_geometry_rules(ora):
    nx, ny = 40, 16
    cells = np.ones((ny, nx), np.uint8)
    cells[0:6, :] = 0  # a channel against the symmetry plane
    p = ora.make_params(nx, ny, 0.8, 1.0, 0.02, mirror=True)
    assert ora.check_geometry(p, cells) == 0
    p0 = ora.make_params(nx, ny, 0.8, 1.0, 0.02)
    assert ora.check_geometry(p0, cells) == 2  # without the plane row 0 must be solid
    # Poiseuille in the half channel: the profile is the upper half of the
    # full parabola across twice the width
    u = ora.inlet_profile(p, cells)
    s = (np.arange(6) + 6 + 0.5) / 12
    np.testing.assert_allclose(u[:6], 4 * 0.02 * s * (1 - s), rtol=1e-15)
