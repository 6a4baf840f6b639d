"""GPU collision models beyond BGK (regularised BGK, Smagorinsky) against
the FP64 oracle, at the FP32 tolerance of the hot path; and the models mixed
with BGK lattices in one batch, each equal bit for bit to its run alone."""
import numpy as np
import pytest

import paper_1303_0107_gb300 as L
from paper_1303_0107_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load_library()


def _block_channel(nx=200, ny=60):
    cells = np.ones((ny, nx), np.uint8)
    cells[1:-1, :] = 0
    cells[22:38, 50:56] = 1
    return cells


def _compare(ora, cells, tau, u_max, steps, collision, c_smag=0.0, tol=TOL, ports=0):
    ny, nx = cells.shape
    lat = L.Lattice(cells, tau, u_max, residual_every=0, collision=collision, c_smag=c_smag, ports=ports)
    g = lat.solve(steps)
    p = ora.make_params(nx, ny, tau, 1.0, u_max, port_scheme=ports, collision=collision, c_smag=c_smag)
    s = ora.Solver(p, cells, residual_every=0)
    o = s.solve(steps)
    ux = lat.read(L.FIELD_UX).astype(np.float64)
    uy = lat.read(L.FIELD_UY).astype(np.float64)
    drho = lat.read(L.FIELD_DRHO).astype(np.float64)
    scale = np.abs(s.ux).max()
    assert np.abs(ux - s.ux).max() <= tol * scale
    assert np.abs(uy - s.uy).max() <= tol * scale
    ref = (s.rho - 1.0) * (cells == 0)
    assert np.abs(drho - ref).max() <= tol * np.abs(ref).max()
    assert abs(g["dp"] - o["dp"]) <= tol * abs(o["dp"])
    lat.close()
    return g


@pytest.mark.parametrize("collision,c_smag", [(L.COLLIDE_REGULARIZED, 0.0), (L.COLLIDE_SMAGORINSKY, 0.1),
                                              (L.COLLIDE_SMAGORINSKY, 0.3)])
@pytest.mark.parametrize("ports", [L.PORTS_REGULARIZED, L.PORTS_ZOU_HE])
def test_models_match_oracle_on_t_junction(ora, collision, c_smag, ports):
    cfg = I.config_t_junction()
    _compare(ora, cfg["cells"], cfg["tau"], cfg["u_max"], 400, collision, c_smag, ports=ports)


def test_smagorinsky_matches_oracle_on_block_channel(ora):
    _compare(ora, _block_channel(), 0.6, 0.05, 600, L.COLLIDE_SMAGORINSKY, 0.15)


def test_smagorinsky_stays_bounded_where_bgk_diverges():
    cells = _block_channel()
    bgk = L.Lattice(cells, 0.51, 0.05, residual_every=0)
    with pytest.raises(L.LbmError) as e:
        for _ in range(4):
            bgk.solve(1000)
    assert e.value.status == 5  # LBM_ERR_DIVERGED
    bgk.close()
    smag = L.Lattice(cells, 0.51, 0.05, residual_every=0, collision=L.COLLIDE_SMAGORINSKY, c_smag=0.1)
    r = smag.solve(4000)
    assert np.isfinite(r["dp"]) and np.abs(smag.read(L.FIELD_UX)).max() < 0.2
    smag.close()


def test_batch_mixing_models_equals_each_alone():
    cfg = I.config_t_junction()
    members = [dict(cells=cfg["cells"], tau=0.8, u_max=0.05),
               dict(cells=cfg["cells"], tau=0.6, u_max=0.04, collision=L.COLLIDE_REGULARIZED),
               dict(cells=_block_channel(), tau=0.55, u_max=0.05, collision=L.COLLIDE_SMAGORINSKY, c_smag=0.12)]
    b = L.Batch(members, residual_every=0)
    rb = b.solve(600)
    ob = b.optimize_step([2, 3, 4], 200)
    assert b.step_config()[2:] == (0, 1, 0)
    for i, m in enumerate(members):
        h = L.Lattice(m["cells"], m["tau"], m["u_max"], residual_every=0, collision=m.get("collision", 0),
                      c_smag=m.get("c_smag", 0.0))
        assert h.solve(600)["dp"] == rb[i]["dp"]
        assert h.optimize_step([2, 3, 4][i], 200)["dp"] == ob[i]["dp"]
        assert np.array_equal(h.read(L.FIELD_POPS), b.read(i, L.FIELD_POPS))
        h.close()
    b.close()


def test_collision_argument_checks():
    cfg = I.config_t_junction()
    for kw in (dict(collision=3), dict(collision=L.COLLIDE_SMAGORINSKY, c_smag=-0.1)):
        with pytest.raises(L.LbmError) as e:
            L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"], **kw)
        assert e.value.status == 1
    h = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"], collision=L.COLLIDE_REGULARIZED)
    with pytest.raises(L.LbmError):  # the models run with the plain launch shape only
        h.set_step_config(8, persistent=True)
    h.close()
