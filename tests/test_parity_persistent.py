"""The persistent stream-collide kernel (all time steps of a solve in one
cooperative launch, grid barriers between phases) against the one-launch-
per-phase kernel and against the FP64 oracle.

Both launch modes run the same per-cell code, so their populations, fields
and reductions must agree bit for bit; the full-size tree is also checked
against the oracle at the FP32 tolerance.
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


def _cases():
    t = I.config_t_junction()
    c = I.config_candidates(1, base_seed=7)[0]
    return [
        dict(cells=t["cells"], tau=t["tau"], u_max=t["u_max"]),
        dict(cells=I.random_blobs(100, 40, 9, density=0.2), tau=0.7, u_max=0.03, outlet=L.OUT_NEUMANN),
        dict(cells=I.channel(64, 14), tau=0.9, u_max=0.04, ports=L.PORTS_ZOU_HE),
        dict(cells=c["cells"], tau=c["tau"], u_max=c["u_max"]),
    ]


def _mirror_case():
    return dict(cells=I.config_collector()["cells"], tau=0.62, u_max=0.12, outlet=L.OUT_NEUMANN, mirror=True)


def _handle(case, precision, persistent, wpb=8, cpt=1, stages=0):
    h = L.Lattice(case["cells"], case["tau"], case["u_max"], precision=precision, outlet=case.get("outlet", 0),
                  ports=case.get("ports", 0), residual_every=100, mirror=case.get("mirror", False))
    h.set_step_config(wpb, persistent=persistent, cells_per_thread=cpt, stages=stages)
    return h


# (persistent, warps per block, cells per thread, shared-memory stages)
SHAPES = [(True, 8, 1, 0), (True, 8, 2, 0), (False, 8, 2, 0), (False, 4, 2, 0), (False, 8, 1, 3), (False, 4, 1, 2),
          (False, 16, 1, 3), (False, 8, 1, 2), (False, 24, 2, 0), (False, 32, 1, 0), (False, 12, 2, 0), (False, 12, 1, 0)]


@pytest.mark.parametrize("precision", [L.F32, L.BF16_SHIFTED, L.F16_SHIFTED])
@pytest.mark.parametrize("k", range(len(SHAPES)))
def test_launch_shapes_compute_the_same_values(k, precision):
    """Each launch shape -- persistent or per-phase, one or two cells per
    thread, loads into registers or staged through shared memory -- against
    the default shape, bit for bit."""
    case = _cases()[k % 4]
    pers, wpb, cpt, stages = SHAPES[k]
    a = _handle(case, precision, False)
    b = _handle(case, precision, pers, wpb=wpb, cpt=cpt, stages=stages)
    cfg = b.step_config()
    assert cfg[2] == int(pers) and cfg[3] == cpt and cfg[4] == stages and a.step_config()[2] == 0
    ra, rb = a.solve(600), b.solve(600)
    assert ra["dp"] == rb["dp"] and ra["residual"] == rb["residual"]
    assert np.array_equal(a.read(L.FIELD_POPS), b.read(L.FIELD_POPS))
    fl = int((case["cells"] == 0).sum())
    oa, ob = a.optimize_step(max(1, fl // 200), 300), b.optimize_step(max(1, fl // 200), 300)
    assert oa["dp"] == ob["dp"] and oa["n_swapped"] == ob["n_swapped"]
    for f in (L.FIELD_MASK, L.FIELD_UX, L.FIELD_UY, L.FIELD_DRHO, L.FIELD_POPS):
        assert np.array_equal(a.read(f), b.read(f)), f
    a.close()
    b.close()


def test_persistent_tree_2048_matches_oracle(ora):
    cfg = I.config_tree_2048()
    cells = cfg["cells"]
    ny, nx = cells.shape
    h = L.Lattice(cells, cfg["tau"], cfg["u_max"], residual_every=0)
    h.set_step_config(8, persistent=True, cells_per_thread=2)
    g = h.solve(300)
    s = ora.Solver(ora.make_params(nx, ny, cfg["tau"], 1.0, cfg["u_max"]), cells, residual_every=0)
    o = s.solve(300)
    ux = h.read(L.FIELD_UX).astype(np.float64)
    uy = h.read(L.FIELD_UY).astype(np.float64)
    assert np.linalg.norm(ux - s.ux) / np.linalg.norm(s.ux) <= 1e-5
    assert np.abs(ux - s.ux).max() / np.abs(s.ux).max() <= 1e-5
    assert np.abs(uy - s.uy).max() / np.abs(s.ux).max() <= 1e-5
    assert abs(g["dp"] - o["dp"]) <= 1e-5 * abs(o["dp"])
    h.close()


@pytest.mark.parametrize("wpb", [4, 16])
def test_feature_builds_keep_values_across_shapes(wpb):
    """Lattices with a symmetry plane or a collision model run the feature
    builds (plain shapes only): every block shape gives the same values, and
    in a batch with plain lattices each member equals its run alone."""
    m = _mirror_case()
    a = _handle(m, L.F32, False)
    b = _handle(m, L.F32, False, wpb=wpb)
    assert a.solve(600)["dp"] == b.solve(600)["dp"]
    assert np.array_equal(a.read(L.FIELD_POPS), b.read(L.FIELD_POPS))
    with pytest.raises(L.LbmError):
        b.set_step_config(8, persistent=True)
    members = _cases()[:2] + [m]
    bt = L.Batch(members, residual_every=0)
    rb = bt.solve(400)
    for i, mm in enumerate(members):
        h = L.Lattice(mm["cells"], mm["tau"], mm["u_max"], outlet=mm.get("outlet", 0), residual_every=0,
                      mirror=mm.get("mirror", False))
        assert h.solve(400)["dp"] == rb[i]["dp"]
        assert np.array_equal(h.read(L.FIELD_POPS), bt.read(i, L.FIELD_POPS)), i
        h.close()
    a.close()
    b.close()
    bt.close()


@pytest.mark.parametrize("shape", [(8, 2, 0), (8, 1, 3)])
def test_batch_shapes_equal_default_batch(shape):
    wpb, cpt, stages = shape
    members = _cases()
    a = L.Batch(members, residual_every=0)
    b = L.Batch(members, residual_every=0)
    a.set_step_config(8, persistent=False)
    b.set_step_config(wpb, persistent=False, cells_per_thread=cpt, stages=stages)
    ra, rb = a.solve(400), b.solve(400)
    assert [x["dp"] for x in ra] == [x["dp"] for x in rb]
    oa, ob = a.optimize_step([3, 2, 1, 4], 200), b.optimize_step([3, 2, 1, 4], 200)
    assert [x["dp"] for x in oa] == [x["dp"] for x in ob]
    for i in range(len(members)):
        assert np.array_equal(a.read(i, L.FIELD_POPS), b.read(i, L.FIELD_POPS)), i
    a.close()
    b.close()


def test_set_step_config_errors():
    t = I.config_t_junction()
    h = L.Lattice(t["cells"], t["tau"], t["u_max"])
    for wpb, pers, cpt, stg in ((3, 0, 1, 0), (64, 0, 1, 0), (24, 0, 1, 0), (32, 0, 2, 0), (4, 1, 1, 0), (8, 5, 1, 0),
                                (8, 0, 3, 0), (16, 0, 2, 0), (24, 1, 2, 0), (32, 1, 1, 0), (32, 0, 1, 2), (8, 1, 0, 0),
                                (8, 0, 1, 1), (8, 0, 1, 4), (8, 1, 1, 2), (8, 0, 2, 3)):
        with pytest.raises(L.LbmError) as e:
            h.set_step_config(wpb, persistent=pers, cells_per_thread=cpt, stages=stg)
        assert e.value.status == 1
    h.close()


def test_barrier_wait_gives_up_and_the_handle_stays_usable():
    """The bounded-wait failure path without a device fault: under the test
    hook every grid barrier waits for one arrival too many, gives up after its
    poll limit, the launch ends early and the solve reports LBM_ERR_TIMEOUT;
    afterwards the context and the handle work as before."""
    import time
    cfg = I.config_t_junction()
    ref = _handle(dict(cells=cfg["cells"], tau=cfg["tau"], u_max=cfg["u_max"]), L.F32, True)
    r_ref = ref.solve(200)
    ref.close()
    h = _handle(dict(cells=cfg["cells"], tau=cfg["tau"], u_max=cfg["u_max"]), L.F32, True)
    L.lib.debug_barrier_timeout(True)
    try:
        t0 = time.perf_counter()
        with pytest.raises(L.LbmError) as e:
            h.solve(200)
        assert e.value.status == 6  # LBM_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 60
    finally:
        L.lib.debug_barrier_timeout(False)
    h.reset()
    assert h.solve(200)["dp"] == r_ref["dp"]
    h.close()


@pytest.mark.parametrize("stages", [0, 2, 3])
@pytest.mark.parametrize("precision", [L.F32, L.BF16_SHIFTED, L.F16_SHIFTED])
@pytest.mark.parametrize("k", [0, 2, 3])
def test_cell_tasks_compute_the_same_values(k, precision, stages):
    """Compacted fluid-cell tasks (32 consecutive fluid cells per warp; their
    populations into registers, or copied into shared memory 1-2 tasks
    ahead) against the default row-segment shape, bit for bit, through
    exchanges (the cell list is rebuilt with the work-list)."""
    case = _cases()[k]
    a = _handle(case, precision, False)
    b = _handle(case, precision, False)
    b.set_step_config(8, persistent=3, stages=stages)
    assert b.step_config()[2] == 3 and b.step_config()[4] == stages
    ra, rb = a.solve(600), b.solve(600)
    assert ra["dp"] == rb["dp"] and ra["residual"] == rb["residual"]
    assert np.array_equal(a.read(L.FIELD_POPS), b.read(L.FIELD_POPS))
    fl = int((case["cells"] == 0).sum())
    for _ in range(2):
        oa, ob = a.optimize_step(max(1, fl // 200), 300), b.optimize_step(max(1, fl // 200), 300)
        assert oa["dp"] == ob["dp"] and oa["n_swapped"] == ob["n_swapped"]
    for f in (L.FIELD_MASK, L.FIELD_UX, L.FIELD_UY, L.FIELD_DRHO, L.FIELD_POPS):
        assert np.array_equal(a.read(f), b.read(f)), f
    a.close()
    b.close()


def test_cell_tasks_in_a_batch_and_where_refused():
    members = [c for c in _cases() if c.get("outlet", 0) == 0]
    a = L.Batch(members, residual_every=0)
    b = L.Batch(members, residual_every=0)
    a.set_step_config(8, persistent=False)
    b.set_step_config(16, persistent=3, stages=3)
    ra, rb = a.solve(400), b.solve(400)
    assert [x["dp"] for x in ra] == [x["dp"] for x in rb]
    n = [3, 1, 4][:len(members)]
    oa, ob = a.optimize_step(n, 200), b.optimize_step(n, 200)
    assert [x["dp"] for x in oa] == [x["dp"] for x in ob]
    for i in range(len(members)):
        assert np.array_equal(a.read(i, L.FIELD_POPS), b.read(i, L.FIELD_POPS)), i
    a.close()
    b.close()
    t = _handle(_cases()[0], L.F32, False)
    for wpb, stg in ((32, 2), (8, 1), (8, 5)):  # 32 warps with stages; stages outside 0, 2-4
        with pytest.raises(L.LbmError) as e:
            t.set_step_config(wpb, persistent=3, stages=stg)
        assert e.value.status == 1
    t.close()
    neumann = _handle(_cases()[1], L.F32, False)  # a zero-gradient outlet: refused
    with pytest.raises(L.LbmError) as e:
        neumann.set_step_config(8, persistent=3)
    assert e.value.status == 1
    neumann.close()
    m = _handle(_mirror_case(), L.F32, False)  # a symmetry plane: refused
    with pytest.raises(L.LbmError):
        m.set_step_config(8, persistent=3)
    m.close()
