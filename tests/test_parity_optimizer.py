"""GPU optimality-criterion step vs the oracle, through the C ABI.

Given the same FP32 field, the choice of cells must be bit-exact: the scores
are FP64 with separately rounded operations on both sides, and ties go to
the smaller cell index.  Over a whole optimisation the GPU's FP32 field
differs from the oracle's FP64 one, so each iteration is checked by feeding
the GPU's own field to the oracle's selector.
"""
import numpy as np
import pytest

import paper_1303_0107_gb300 as L
from paper_1303_0107_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load_library()


def _oracle_pick(ora, p, cells, drho, ux, uy, n):
    rho = 1.0 + drho.astype(np.float64)
    cand, score = ora.scores(p, cells, rho, ux.astype(np.float64), uy.astype(np.float64))
    return ora.select(p, cand, score, n)


@pytest.mark.parametrize("seed", range(6))
def test_selection_bit_exact_random_fields(ora, seed):
    cfg = I.config_t_junction()
    cells = cfg["cells"]
    rng = np.random.default_rng(seed)
    shape = cells.shape
    drho = (0.01 * rng.standard_normal(shape)).astype(np.float32)
    ux = (0.05 * rng.standard_normal(shape)).astype(np.float32)
    uy = (0.05 * rng.standard_normal(shape)).astype(np.float32)
    if seed % 2:  # quantised values: exact ties everywhere
        ux = (np.round(ux * 40) / 40).astype(np.float32)
        uy = (np.round(uy * 40) / 40).astype(np.float32)
        drho[:] = 0
    lat = L.Lattice(cells, cfg["tau"], cfg["u_max"])
    p = ora.make_params(128, 64, cfg["tau"], 1.0, cfg["u_max"])
    for n in (0, 1, 2, 7, 64, 100000):
        fi, si = lat.select_swaps(drho, ux, uy, n)
        fo, so = _oracle_pick(ora, p, cells, drho, ux, uy, n)
        assert np.array_equal(fi, fo) and np.array_equal(si, so), n


def test_selection_bit_exact_ragged_random_masks(ora):
    for seed in range(4):
        nx, ny = [(40, 12), (70, 33), (98, 20), (130, 17)][seed]
        cells = I.random_blobs(nx, ny, seed + 10, density=0.3)
        rng = np.random.default_rng(seed)
        f = [(0.02 * rng.standard_normal((ny, nx))).astype(np.float32) for _ in range(3)]
        lat = L.Lattice(cells, 0.7, 0.02)
        p = ora.make_params(nx, ny, 0.7, 1.0, 0.02)
        for n in (1, 5, 50):
            fi, si = lat.select_swaps(*f, n)
            fo, so = _oracle_pick(ora, p, cells, *f, n)
            assert np.array_equal(fi, fo) and np.array_equal(si, so)


def test_optimisation_loop_matches_oracle_choice(ora):
    """Ten iterations of the 128 x 64 T-junction loop (exchange 2 cells, 2000
    steps).  Each iteration: the GPU's exchange equals the oracle's pick on the
    GPU field; the oracle is restarted from the GPU's populations, makes the
    same exchange and re-solves, and the two pressure drops agree to the FP32
    bar of one solve (1e-5); the fluid count never changes."""
    W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    cfg = I.config_t_junction()
    cells = cfg["cells"]
    lat = L.Lattice(cells, cfg["tau"], cfg["u_max"])
    p = ora.make_params(128, 64, cfg["tau"], 1.0, cfg["u_max"])
    s = ora.Solver(p, cells)
    lat.solve(cfg["steps"])
    n0 = int((cells == 0).sum())
    worst = 0.0
    for it in range(cfg["n_iter"]):
        drho, ux, uy = (lat.read(L.FIELD_DRHO), lat.read(L.FIELD_UX), lat.read(L.FIELD_UY))
        mask_before = lat.read(L.FIELD_MASK)
        fo, so = _oracle_pick(ora, p, mask_before, drho, ux, uy, 2)
        s.solid = mask_before.copy()
        s.f = lat.read(L.FIELD_POPS).astype(np.float64) + W[:, None, None]
        r = lat.optimize_step(2, cfg["steps"])
        assert r["n_swapped"] == len(fo) == 2
        assert r["fluid_count"] == n0
        expect = mask_before.copy().reshape(-1)
        expect[fo] = 1
        expect[so] = 0
        assert np.array_equal(lat.read(L.FIELD_MASK).reshape(-1), expect)
        s.exchange(fo, so)
        o = s.solve(cfg["steps"])
        rel = abs(r["dp"] - o["dp"]) / abs(o["dp"])
        worst = max(worst, rel)
        assert rel <= 1e-5, (it, rel)
    print(f"worst per-solve relative dp difference over the loop: {worst:.2e}")
    assert int((lat.read(L.FIELD_MASK) == 0).sum()) == n0


def test_exchange_reinitialises_new_fluid_cells(ora):
    cfg = I.config_t_junction()
    lat = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"])
    lat.solve(500)
    drho, ux, uy = (lat.read(L.FIELD_DRHO), lat.read(L.FIELD_UX), lat.read(L.FIELD_UY))
    fi, si = lat.select_swaps(drho, ux, uy, 4)
    # run the exchange with the shortest re-solve, then inspect populations of
    # the new fluid cells right after 2 more steps is not possible; instead
    # compare with the oracle doing the same exchange from the GPU state
    pops = lat.read(L.FIELD_POPS).astype(np.float64)
    W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    p = ora.make_params(128, 64, cfg["tau"], 1.0, cfg["u_max"])
    s = ora.Solver(p, cfg["cells"])
    s.f = pops + W[:, None, None]
    s.rho, s.ux, s.uy = 1.0 + drho.astype(np.float64), ux.astype(np.float64), uy.astype(np.float64)
    fo, so = s.pick(4)
    assert np.array_equal(fo, fi) and np.array_equal(so, si)
    s.exchange(fo, so)
    r = lat.optimize_step(4, 2)
    o = s.solve(2)
    assert abs(r["dp"] - o["dp"]) <= 1e-5 * abs(o["dp"])
    f_gpu = lat.read(L.FIELD_POPS).astype(np.float64) + W[:, None, None]
    fluid = s.solid == 0
    assert np.abs(f_gpu - s.f)[:, fluid].max() <= 4e-6 * W.max()


def test_cold_reinit(ora):
    cfg = I.config_t_junction()
    lat = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"], reinit=L.REINIT_COLD)
    lat.solve(300)
    drho, ux, uy = (lat.read(L.FIELD_DRHO), lat.read(L.FIELD_UX), lat.read(L.FIELD_UY))
    p = ora.make_params(128, 64, cfg["tau"], 1.0, cfg["u_max"])
    s = ora.Solver(p, cfg["cells"], reinit=ora.REINIT_COLD)
    s.rho, s.ux, s.uy = 1.0 + drho.astype(np.float64), ux.astype(np.float64), uy.astype(np.float64)
    fo, so = s.pick(3)
    s.exchange(fo, so)  # every fluid cell back to rest
    r = lat.optimize_step(3, 200)
    o = s.solve(200)
    assert abs(r["dp"] - o["dp"]) <= 1e-5 * abs(o["dp"])


@pytest.mark.parametrize("seed", range(4))
def test_guarded_selection_bit_exact(ora, seed):
    """The connectivity guard on the GPU (word-parallel 4-connectivity
    numbers) against the oracle's cell-by-cell rule, on ragged random masks
    with thin walls and necks."""
    nx, ny = [(64, 24), (70, 33), (130, 17), (256, 40)][seed]
    cells = I.random_blobs(nx, ny, seed + 30, density=0.35)
    rng = np.random.default_rng(seed + 5)
    f = [(0.02 * rng.standard_normal((ny, nx))).astype(np.float32) for _ in range(3)]
    lat = L.Lattice(cells, 0.7, 0.02, guard=True)
    p = ora.make_params(nx, ny, 0.7, 1.0, 0.02, guard=True)
    p0 = ora.make_params(nx, ny, 0.7, 1.0, 0.02)
    for n in (1, 5, 50, 100000):
        fi, si = lat.select_swaps(*f, n)
        fo, so = _oracle_pick(ora, p, cells, *f, n)
        assert np.array_equal(fi, fo) and np.array_equal(si, so), (seed, n)
    # the guard removes candidates: the unguarded choice of all candidates is larger
    fu, _ = _oracle_pick(ora, p0, cells, *f, 100000)
    assert len(fu) >= len(fi)


def test_guarded_loop_keeps_the_channel_connected(ora):
    """Many aggressive exchanges on the T-junction: with the guard every
    iteration's mask keeps a single 4-connected fluid region."""
    from test_oracle_optimizer import _components
    cfg = I.config_t_junction()
    lat = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"], residual_every=0, guard=True)
    lat.solve(400)
    for _ in range(12):
        r = lat.optimize_step(12, 200)
        mask = lat.read(L.FIELD_MASK)
        assert _components(mask == 0) == 1
        assert r["fluid_count"] == int((cfg["cells"] == 0).sum())
    lat.close()
