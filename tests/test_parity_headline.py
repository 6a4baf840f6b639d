"""The benchmark configuration itself against the FP64 oracle, through the C ABI.

The 2048 x 1024 four-generation distributor (widths 64/32/16/8/4, jitter
+-2, seed 0, tau 0.53, u_max 0.01171875) is solved for 5000 time steps --
one solve of the optimisation run of Sec. 2.3 -- by a handle created exactly
as the benchmark creates it (the launch shape is the one the engine's tuner
picks at the first solve), then:
  * the fields rho - rho0, u_x, u_y (L2 and max norm), the pressure drop,
    the inlet flow rate and every outlet flow rate within 1e-5 of the oracle;
  * the exchange of the benchmark (n_swap = 0.2 % of the fluid = 319 cells
    each way) chosen on the GPU's own field bit for bit as the oracle's
    selection on that field, and the cell map after one optimiser step
    equal to the oracle applying the same picks.

The oracle takes ~16 s for the 5000 steps on 16 cores.

The convergence residual (Sec. 2.3 step 5) is checked here too: the GPU's
FP64 reduction against the same ratio formed on the host from the GPU's own
FP32 fields at T - K and T (1e-12), and against the oracle within the bound
the field errors imply.  The residual divides the difference of two nearly
equal fields by their size, so an error e in each field (relative, L1) moves
r by at most (1 + r) e_T + e_(T-K): a fixed relative bar of 1e-5 on r
itself would ask for field errors r times smaller than the field bar.
"""
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


def _l1(ux, uy, fluid):
    return np.abs(ux)[fluid].sum() + np.abs(uy)[fluid].sum()


@pytest.fixture(scope="module")
def headline(ora):
    cfg = I.config_tree_2048()
    cells = cfg["cells"]
    ny, nx = cells.shape
    S = cfg["steps"]
    lat = L.Lattice(cells, cfg["tau"], cfg["u_max"], residual_every=100)
    g = lat.solve(S)
    s = ora.Solver(ora.make_params(nx, ny, cfg["tau"], 1.0, cfg["u_max"]), cells, residual_every=100)
    o = s.solve(S)
    yield cfg, lat, g, s, o
    lat.close()


def test_headline_solve_fields_and_flow_rates(headline):
    cfg, lat, g, s, o = headline
    cells = cfg["cells"]
    fluid = cells == 0
    drho = lat.read(L.FIELD_DRHO).astype(np.float64)
    ux = lat.read(L.FIELD_UX).astype(np.float64)
    uy = lat.read(L.FIELD_UY).astype(np.float64)
    ref = {"drho": (s.rho - 1.0) * fluid, "ux": s.ux, "uy": s.uy}
    got = {"drho": drho, "ux": ux, "uy": uy}
    uscale2 = max(np.linalg.norm(s.ux), np.linalg.norm(s.uy))
    uscale = max(np.abs(s.ux).max(), np.abs(s.uy).max())
    for k in got:
        d = got[k] - ref[k]
        s2 = uscale2 if k == "uy" else np.linalg.norm(ref[k])
        sm = uscale if k == "uy" else np.abs(ref[k]).max()
        assert np.linalg.norm(d) <= TOL * s2, (k, np.linalg.norm(d) / s2)
        assert np.abs(d).max() <= TOL * sm, (k, np.abs(d).max() / sm)
    assert abs(g["dp"] - o["dp"]) <= TOL * abs(o["dp"])
    assert abs(g["m_in"] - o["m_in"]) <= TOL * abs(o["m_in"])
    assert g["n_outlets"] == len(o["m_out"]) == 16
    m_g, m_o = np.asarray(g["m_out"]), np.asarray(o["m_out"])
    # after 5000 steps every outlet carries flow: each within 1e-5 of itself
    assert np.all(m_o > 0)
    assert np.all(np.abs(m_g - m_o) <= TOL * np.abs(m_o)), np.abs(m_g - m_o) / np.abs(m_o)
    assert g["theta"] == pytest.approx(o["theta"], rel=2 * TOL)
    assert abs(g["dg"] - o["dg"]) <= 2 * TOL
    assert g["fluid_cells"] == int(fluid.sum()) == 159872


def test_headline_exchange_of_319_cells_bit_exact(headline, ora):
    cfg, lat, g, s, o = headline
    cells = cfg["cells"]
    n_swap = max(1, int(0.002 * int((cells == 0).sum())))
    assert n_swap == 319
    drho = lat.read(L.FIELD_DRHO)
    ux = lat.read(L.FIELD_UX)
    uy = lat.read(L.FIELD_UY)
    rho = 1.0 + drho.astype(np.float64)
    fi_o, si_o = s.pick(n_swap, rho=rho, ux=ux.astype(np.float64), uy=uy.astype(np.float64))
    assert len(fi_o) == len(si_o) == n_swap
    fi_g, si_g = lat.select_swaps(drho, ux, uy, n_swap)
    assert np.array_equal(np.asarray(fi_g), np.asarray(fi_o))
    assert np.array_equal(np.asarray(si_g), np.asarray(si_o))
    # the optimiser step chooses from the handle's own last field: the same picks
    r = lat.optimize_step(n_swap, 2)
    assert r["n_swapped"] == n_swap and r["fluid_count"] == 159872
    s.exchange(fi_o, si_o)
    assert np.array_equal(lat.read(L.FIELD_MASK), s.solid)


def test_residual_reduction_and_bound(ora):
    """T = 2000, K = 100 on the 128 x 64 T-junction (tau 0.8, u_max 0.05)."""
    cfg = I.config_t_junction()
    cells = cfg["cells"]
    ny, nx = cells.shape
    fluid = cells == 0
    K, T = 100, cfg["steps"]
    one = L.Lattice(cells, cfg["tau"], cfg["u_max"], residual_every=K)
    r_gpu = one.solve(T)["residual"]
    one.close()
    two = L.Lattice(cells, cfg["tau"], cfg["u_max"], residual_every=0)
    two.solve(T - K)
    uxp = two.read(L.FIELD_UX).astype(np.float64)
    uyp = two.read(L.FIELD_UY).astype(np.float64)
    two.solve(K)
    ux = two.read(L.FIELD_UX).astype(np.float64)
    uy = two.read(L.FIELD_UY).astype(np.float64)
    two.close()
    # the GPU's reduction on its own fields (a continued solve is bit-identical)
    r_host = _l1(ux - uxp, uy - uyp, fluid) / _l1(ux, uy, fluid)
    assert r_gpu == pytest.approx(r_host, rel=1e-12)
    # against the oracle, within the bound the field errors imply
    p = ora.make_params(nx, ny, cfg["tau"], 1.0, cfg["u_max"])
    u_in = ora.inlet_profile(p, cells)
    f = ora.init(p, cells)
    f, _, oxp, oyp, _ = ora.run(p, cells, u_in, f, T - K)
    _, _, ox, oy, _ = ora.run(p, cells, u_in, f, K)
    r_ora = ora.residual(p, cells, ox, oy, oxp, oyp)
    # r_g - r_o = (N_g - N_o) / D_g + r_o (D_o - D_g) / D_g, with
    # |N_g - N_o| <= E_T + E_(T-K) and |D_g - D_o| <= E_T (E: L1 field errors)
    den_g = _l1(ux, uy, fluid)
    e_t = _l1(ux - ox, uy - oy, fluid) / den_g
    e_tk = _l1(uxp - oxp, uyp - oyp, fluid) / den_g
    assert e_t <= TOL and e_tk <= TOL
    bound = (1.0 + r_ora) * e_t + e_tk
    assert abs(r_gpu - r_ora) <= bound + 1e-12, (r_gpu, r_ora, bound)
    print(f"residual gpu {r_gpu:.9e} oracle {r_ora:.9e} bound {bound:.2e}")
