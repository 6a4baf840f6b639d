"""On-chip resident time steps (a whole solve in one launch, the populations
in shared memory, neighbouring blocks exchanging tagged halo words through
global memory) against the one-launch-per-phase kernel, bit for bit, and
against the FP64 oracle on the benchmark lattice.

The resident kernel runs the same per-cell update as the other step
kernels, so every field, population and reduction must agree to the bit:
on one block (the 128 x 64 T), on tens of blocks with obstacles, a ragged
odd-width lattice with the zero-gradient outlet, and the 2048 x 1024 tree
(146 blocks); through exchanges (the work-list, and so the partition,
changes) and in a batch of several lattices.
"""
import numpy as np
import pytest

import paper_1303_0107_gb300 as L
from paper_1303_0107_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RESIDENT = 2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load_library()


def _cases():
    t = I.config_t_junction()
    c = I.config_candidates(1, base_seed=3)[0]
    return [
        dict(cells=t["cells"], tau=t["tau"], u_max=t["u_max"]),
        dict(cells=I.random_blobs(256, 130, 11, density=0.2), tau=0.7, u_max=0.03),
        dict(cells=I.random_blobs(95, 61, 12, density=0.15), tau=0.75, u_max=0.03, outlet=L.OUT_NEUMANN),
        dict(cells=I.channel(64, 14), tau=0.9, u_max=0.04, ports=L.PORTS_ZOU_HE),
        dict(cells=c["cells"], tau=c["tau"], u_max=c["u_max"]),
    ]


def _handle(case, precision, resident):
    h = L.Lattice(case["cells"], case["tau"], case["u_max"], precision=precision, outlet=case.get("outlet", 0),
                  ports=case.get("ports", 0), residual_every=100)
    if resident:
        h.set_step_config(8, persistent=RESIDENT)
        assert h.step_config()[2] == RESIDENT
    else:
        h.set_step_config(8, persistent=False)
    return h


def _same(a, b, members=None):
    for f in (L.FIELD_MASK, L.FIELD_UX, L.FIELD_UY, L.FIELD_DRHO, L.FIELD_POPS):
        assert np.array_equal(a.read(f), b.read(f)), f


@pytest.mark.parametrize("precision", [L.F32, L.BF16_SHIFTED, L.F16_SHIFTED])
@pytest.mark.parametrize("k", range(5))
def test_resident_equals_per_phase_kernel(k, precision):
    case = _cases()[k]
    a = _handle(case, precision, False)
    b = _handle(case, precision, True)
    ra, rb = a.solve(600), b.solve(600)
    assert ra["dp"] == rb["dp"] and ra["residual"] == rb["residual"] and ra["m_in"] == rb["m_in"]
    assert list(ra["m_out"]) == list(rb["m_out"])
    _same(a, b)
    fl = int((case["cells"] == 0).sum())
    for it in range(2):  # the exchange rebuilds the work-list: a new partition each time
        oa, ob = a.optimize_step(max(1, fl // 200), 300), b.optimize_step(max(1, fl // 200), 300)
        assert oa["dp"] == ob["dp"] and oa["n_swapped"] == ob["n_swapped"]
        _same(a, b)
    assert b.step_config()[2] == RESIDENT
    a.close()
    b.close()


def test_resident_tree_2048_bit_equal_and_against_oracle(ora):
    cfg = I.config_tree_2048()
    cells = cfg["cells"]
    ny, nx = cells.shape
    case = dict(cells=cells, tau=cfg["tau"], u_max=cfg["u_max"])
    a = _handle(case, L.F32, False)
    b = _handle(case, L.F32, True)
    w, grid, pers, cpt, stages = b.step_config()
    assert pers == RESIDENT and grid == 146 and 1 <= w <= 24
    assert a.solve(300)["dp"] == b.solve(300)["dp"]
    _same(a, b)
    s = ora.Solver(ora.make_params(nx, ny, cfg["tau"], 1.0, cfg["u_max"]), cells, residual_every=0)
    o = s.solve(300)
    ux = b.read(L.FIELD_UX).astype(np.float64)
    assert np.abs(ux - s.ux).max() <= 1e-5 * np.abs(s.ux).max()
    assert a.solve(2)["dp"] == b.solve(2)["dp"]  # continued from the state written back
    _same(a, b)
    a.close()
    b.close()


def test_resident_batch_members_equal_their_runs_alone():
    members = _cases()
    bt = L.Batch(members, residual_every=0)
    bt.set_step_config(8, persistent=RESIDENT)
    assert bt.step_config()[2] == RESIDENT
    rb = bt.solve(400)
    ob = bt.optimize_step([3, 4, 2, 1, 5], 200)
    for i, m in enumerate(members):
        h = L.Lattice(m["cells"], m["tau"], m["u_max"], outlet=m.get("outlet", 0), ports=m.get("ports", 0),
                      residual_every=0)
        h.set_step_config(8, persistent=False)
        assert h.solve(400)["dp"] == rb[i]["dp"]
        assert h.optimize_step([3, 4, 2, 1, 5][i], 200)["dp"] == ob[i]["dp"]
        assert np.array_equal(h.read(L.FIELD_POPS), bt.read(i, L.FIELD_POPS)), i
        h.close()
    bt.close()


def test_resident_refused_where_it_cannot_run():
    big = I.channel_array(8192, 4096, 16, fill=0.5)  # ~130 000 segments: more than the SMs hold
    h = L.Lattice(big, 0.6, 0.05, residual_every=0)
    with pytest.raises(L.LbmError) as e:
        h.set_step_config(8, persistent=RESIDENT)
    assert e.value.status == 1
    h.close()
    col = I.config_collector()  # a symmetry plane: the feature build only
    m = L.Lattice(col["cells"], col["tau"], col["u_max"], mirror=True)
    with pytest.raises(L.LbmError):
        m.set_step_config(8, persistent=RESIDENT)
    m.close()


def test_resident_wait_gives_up_and_the_handle_stays_usable():
    """Under the test hook every halo wait expects a tag that nobody writes:
    each block gives up after its poll limit (or when it sees another block's
    error word), the solve reports LBM_ERR_TIMEOUT, and after a reset the
    same handle reproduces its reference pressure drop."""
    import time
    case = _cases()[1]
    ref = _handle(case, L.F32, True)
    r_ref = ref.solve(200)
    ref.close()
    h = _handle(case, L.F32, True)
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
