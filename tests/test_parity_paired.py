"""Paired tasks (launch mode 4): interior windows of 64 cells taken two cells
a lane with paired loads and stores, every other row segment as in the
default shape, in one launch per phase; the windows' pairs loaded into
registers or copied into shared memory tasks ahead (stages).

* The window count of the task list against a host-side count from the
  cell map (row y, cells 64p .. 64p+63 with rows y-1..y+1 fluid over cells
  64p-1 .. 64p+64).  This shows that the paired path is taken and where.
* Populations, fields and reductions bit for bit against the default shape,
  at FP32, BF16 and FP16, through solves and exchanges (the list is rebuilt
  with the work-list).  The lattices put window edges next to walls, give
  rows an odd number of mask words, and have both outlet rules.
* Against the FP64 oracle at the FP32 tolerance.
* In a batch, and the refusals.
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


def interior_windows(cells):
    """Host count of interior windows: for every row y in 1..ny-2 and window
    p (mask words 2p and 2p+1 both inside the row, i.e. 2p + 1 < wpr),
    cells 64p-1 .. 64p+64 of rows y-1..y+1 are fluid (columns outside
    0..nx-1 count as solid)."""
    ny, nx = cells.shape
    wpr = (nx + 31) // 32
    width = 64 * ((wpr + 1) // 2) + 2
    solid = np.ones((ny, width), bool)
    solid[:, 1:nx + 1] = cells != 0  # column x at index x + 1
    n = 0
    for p in range(wpr // 2):
        bad = solid[:, 64 * p:64 * p + 66].any(axis=1)
        n += int((~(bad[:-2] | bad[1:-1] | bad[2:])).sum())
    return n


def fluid_segments(cells):
    ny, nx = cells.shape
    wpr = (nx + 31) // 32
    fl = np.zeros((ny, 32 * wpr), bool)
    fl[:, :nx] = cells == 0
    return int(fl[1:ny - 1].reshape(ny - 2, wpr, 32).any(axis=2).sum())


def _walls_case():
    """Three wide channels over 1000 columns (32 mask words a row, the last
    one partly past the lattice), with single solid cells on a window's west
    edge (x = 63), on its east edge (x = 128) and inside one (x = 300)."""
    cells = I.channel_array(1000, 150, 3, fill=0.6)
    mid = 25
    cells[mid, 63] = 1
    cells[mid + 5, 128] = 1
    cells[mid + 10, 300] = 1
    cells[75, 640] = 1
    return dict(cells=cells, tau=0.6, u_max=0.05)


def _cases():
    return [
        _walls_case(),
        # 968 columns: 31 mask words a row (the last window would reach the padding word)
        dict(cells=I.channel(968, 40), tau=0.7, u_max=0.04, outlet=L.OUT_NEUMANN),
        dict(cells=I.tree(768, 384, 3, 48), tau=0.6, u_max=0.05),
        dict(cells=I.random_blobs(300, 80, 5, density=0.003), tau=0.8, u_max=0.04, ports=L.PORTS_ZOU_HE),
    ]


def _handle(case, precision):
    return L.Lattice(case["cells"], case["tau"], case["u_max"], precision=precision, outlet=case.get("outlet", 0),
                     ports=case.get("ports", 0), residual_every=100)


@pytest.mark.parametrize("k", range(4))
def test_window_count_matches_the_cell_map(k):
    case = _cases()[k]
    h = _handle(case, L.F32)
    seg, win = h.task_counts()
    assert seg == fluid_segments(case["cells"])
    assert win == interior_windows(case["cells"])
    if k in (0, 1, 2):
        assert win > 0
    h.close()


def test_window_count_after_an_exchange():
    case = _walls_case()
    h = _handle(case, L.F32)
    h.solve(200)
    h.optimize_step(40, 100)
    mask = h.read(L.FIELD_MASK)
    seg, win = h.task_counts()
    assert seg == fluid_segments(mask) and win == interior_windows(mask)
    h.close()


@pytest.mark.parametrize("stages", [0, 3])
@pytest.mark.parametrize("precision", [L.F32, L.BF16_SHIFTED, L.F16_SHIFTED])
@pytest.mark.parametrize("k", range(4))
def test_paired_tasks_compute_the_same_values(k, precision, stages):
    """stages 0: windows loaded into registers; 3: copied into shared
    memory two tasks ahead.  A single lattice takes the kernels with its
    descriptor as a parameter; the batch test below the table-reading ones."""
    case = _cases()[k]
    a = _handle(case, precision)
    b = _handle(case, precision)
    a.set_step_config(8, persistent=False)
    b.set_step_config(8, persistent=4, cells_per_thread=2, stages=stages)
    assert b.step_config()[2] == 4 and b.step_config()[3] == 2 and b.step_config()[4] == stages
    ra, rb = a.solve(600), b.solve(600)
    assert ra["dp"] == rb["dp"] and ra["residual"] == rb["residual"]
    assert np.array_equal(ra["m_out"], rb["m_out"])
    assert np.array_equal(a.read(L.FIELD_POPS), b.read(L.FIELD_POPS))
    fl = int((case["cells"] == 0).sum())
    for _ in range(2):
        oa, ob = a.optimize_step(max(1, fl // 200), 300), b.optimize_step(max(1, fl // 200), 300)
        assert oa["dp"] == ob["dp"] and oa["n_swapped"] == ob["n_swapped"]
    for f in (L.FIELD_MASK, L.FIELD_UX, L.FIELD_UY, L.FIELD_DRHO, L.FIELD_POPS):
        assert np.array_equal(a.read(f), b.read(f)), f
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [L.F32, L.BF16_SHIFTED])
@pytest.mark.parametrize("wpb,stages", [(4, 0), (12, 0), (24, 0), (4, 2), (12, 3), (24, 3), (8, 4), (24, 4)])
def test_block_shapes_compute_the_same_values(wpb, stages, precision):
    case = _walls_case()
    a = _handle(case, precision)
    b = _handle(case, precision)
    a.set_step_config(8, persistent=4, cells_per_thread=2)
    b.set_step_config(wpb, persistent=4, cells_per_thread=2, stages=stages)
    ra, rb = a.solve(400), b.solve(400)
    assert ra["dp"] == rb["dp"]
    assert np.array_equal(a.read(L.FIELD_POPS), b.read(L.FIELD_POPS))
    a.close()
    b.close()


def test_paired_tasks_match_oracle(ora):
    case = _walls_case()
    cells = case["cells"]
    ny, nx = cells.shape
    h = L.Lattice(cells, case["tau"], case["u_max"], residual_every=0)
    h.set_step_config(8, persistent=4, cells_per_thread=2, stages=3)
    g = h.solve(400)
    s = ora.Solver(ora.make_params(nx, ny, case["tau"], 1.0, case["u_max"]), cells, residual_every=0)
    o = s.solve(400)
    ux = h.read(L.FIELD_UX).astype(np.float64)
    uy = h.read(L.FIELD_UY).astype(np.float64)
    assert np.linalg.norm(ux - s.ux) / np.linalg.norm(s.ux) <= 1e-5
    assert np.abs(ux - s.ux).max() / np.abs(s.ux).max() <= 1e-5
    assert np.abs(uy - s.uy).max() / np.abs(s.ux).max() <= 1e-5
    assert abs(g["dp"] - o["dp"]) <= 1e-5 * abs(o["dp"])
    h.close()


def test_paired_tasks_in_a_batch_and_where_refused():
    members = _cases()
    a = L.Batch(members, residual_every=0)
    b = L.Batch(members, residual_every=0)
    a.set_step_config(8, persistent=False)
    b.set_step_config(12, persistent=4, cells_per_thread=2, stages=3)
    ra, rb = a.solve(400), b.solve(400)
    assert [x["dp"] for x in ra] == [x["dp"] for x in rb]
    n = [5, 2, 7, 3]
    oa, ob = a.optimize_step(n, 200), b.optimize_step(n, 200)
    assert [x["dp"] for x in oa] == [x["dp"] for x in ob]
    for i in range(len(members)):
        assert np.array_equal(a.read(i, L.FIELD_POPS), b.read(i, L.FIELD_POPS)), i
    a.close()
    b.close()
    h = _handle(_walls_case(), L.F32)
    # block shapes the paired kernel does not take
    for wpb, cpt, stg in ((16, 2, 0), (32, 2, 0), (8, 1, 0), (8, 2, 1), (8, 2, 5), (8, 2, -1)):
        with pytest.raises(L.LbmError) as e:
            h.set_step_config(wpb, persistent=4, cells_per_thread=cpt, stages=stg)
        assert e.value.status == 1
    h.close()
    m = L.Lattice(I.config_collector()["cells"], 0.62, 0.12, outlet=L.OUT_NEUMANN, mirror=True)
    with pytest.raises(L.LbmError):  # a symmetry plane: the feature build, refused
        m.set_step_config(8, persistent=4, cells_per_thread=2)
    m.close()
    t = I.config_t_junction()
    c = L.Lattice(t["cells"], t["tau"], t["u_max"], collision=L.COLLIDE_SMAGORINSKY, c_smag=0.1)
    with pytest.raises(L.LbmError):  # a collision model beyond BGK: refused
        c.set_step_config(8, persistent=4, cells_per_thread=2)
    c.close()
