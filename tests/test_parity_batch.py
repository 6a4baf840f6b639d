"""Batches: many lattices stepped by one launch per stage.

Every member of a batch must evolve exactly as it does in a handle of its own
-- the per-cell arithmetic and the per-lattice reductions are the same, so the
results are equal bit for bit -- and one member is spot-checked against the
FP64 oracle at the stated FP32 tolerance.
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


def _members():
    t = I.config_t_junction()
    cand = I.config_candidates(3, base_seed=40)
    return [
        dict(cells=t["cells"], tau=t["tau"], u_max=t["u_max"]),
        dict(cells=cand[0]["cells"], tau=cand[0]["tau"], u_max=cand[0]["u_max"]),
        dict(cells=I.random_blobs(100, 40, 9, density=0.2), tau=0.7, u_max=0.03, outlet=L.OUT_NEUMANN),
        dict(cells=cand[1]["cells"], tau=0.6, u_max=0.02, ports=L.PORTS_ZOU_HE),
        dict(cells=I.channel(64, 14), tau=0.9, u_max=0.04, reinit=L.REINIT_COLD),
    ]


def test_batch_members_equal_single_handles_bitwise():
    members = _members()
    batch = L.Batch(members, residual_every=100)
    rb = batch.solve(600)
    singles = [L.Lattice(m["cells"], m["tau"], m["u_max"], outlet=m.get("outlet", 0), ports=m.get("ports", 0),
                         reinit=m.get("reinit", 0), residual_every=100) for m in members]
    for i, (m, h) in enumerate(zip(members, singles)):
        rs = h.solve(600)
        assert rb[i]["dp"] == rs["dp"] and rb[i]["residual"] == rs["residual"], i
        assert np.array_equal(rb[i]["m_out"], rs["m_out"])
        for fld in (L.FIELD_UX, L.FIELD_UY, L.FIELD_DRHO):
            assert np.array_equal(batch.read(i, fld), h.read(fld)), (i, fld)
    # an exchange with a different count per member, then the same on handles
    n_swap = [2, 5, 3, 0, 4]
    ob = batch.optimize_step(n_swap, 200)
    for i, h in enumerate(singles):
        os_ = h.optimize_step(n_swap[i], 200)
        assert ob[i]["n_swapped"] == os_["n_swapped"]
        assert ob[i]["fluid_count"] == os_["fluid_count"] == int((members[i]["cells"] == 0).sum())
        assert ob[i]["dp"] == os_["dp"], i
        assert np.array_equal(batch.read(i, L.FIELD_MASK), h.read(L.FIELD_MASK))
        h.close()
    w, g, _, _, _ = batch.step_config()
    assert w in (4, 8, 16) and g >= 1
    batch.close()


def test_batch_member_matches_oracle(ora):
    members = _members()
    batch = L.Batch(members, residual_every=0)
    rb = batch.solve(400)
    m = members[2]  # irregular walls, zero-gradient outlet
    ny, nx = m["cells"].shape
    p = ora.make_params(nx, ny, m["tau"], 1.0, m["u_max"], ora.OUT_NEUMANN)
    s = ora.Solver(p, m["cells"], residual_every=0)
    o = s.solve(400)
    ux = batch.read(2, L.FIELD_UX).astype(np.float64)
    assert np.linalg.norm(ux - s.ux) / np.linalg.norm(s.ux) <= 1e-5
    assert abs(rb[2]["dp"] - o["dp"]) <= 1e-5 * abs(o["dp"])


def test_batch_reset_and_errors():
    members = _members()[:2]
    batch = L.Batch(members)
    r1 = batch.solve(100)
    batch.optimize_step([3, 3], 100)
    batch.reset()
    r2 = batch.solve(100)
    assert [a["dp"] for a in r1] == [b["dp"] for b in r2]
    with pytest.raises(L.LbmError):
        batch.read(5, L.FIELD_UX)
    with pytest.raises(L.LbmError):
        L.Batch([dict(cells=I.channel(33, 8), tau=0.8, u_max=0.01, outlet=L.OUT_NEUMANN)])
    batch.close()


def test_member_groups_equal_the_ungrouped_batch(monkeypatch):
    """A batch whose populations exceed the group budget runs its time steps
    in member groups (each with its own work-list and tuned shape); every
    member's populations, fields and reductions equal those of the same
    batch stepped as one set with a fixed shape, bit for bit, through
    solves with the residual and through exchanges (the groups' lists are
    rebuilt with the batch's)."""
    cands = [c for c in I.config_candidates(80, base_seed=40) if int((c["cells"] == 0).sum()) < 25000][:14]
    members = [dict(cells=c["cells"], tau=c["tau"], u_max=c["u_max"]) for c in cands]
    fluid = [int((c["cells"] == 0).sum()) for c in cands]
    budget = 4 * 9 * 4 * max(fluid)  # FP32 population bytes of four of the largest members
    assert 9 * 4 * sum(fluid) > 1.5 * budget
    monkeypatch.setenv("LBM_GROUP_BYTES", str(budget))
    a = L.Batch(members, residual_every=100)
    b = L.Batch(members, residual_every=100)
    b.set_step_config(8, persistent=False)
    ra, rb = a.solve(400), b.solve(400)
    assert a.step_groups() > 1 and b.step_groups() == 1
    assert [x["dp"] for x in ra] == [x["dp"] for x in rb]
    assert [x["residual"] for x in ra] == [x["residual"] for x in rb]
    n = [max(1, f // 400) for f in fluid]
    for _ in range(2):
        oa, ob = a.optimize_step(n, 300), b.optimize_step(n, 300)
        assert [x["dp"] for x in oa] == [x["dp"] for x in ob]
        assert [x["n_swapped"] for x in oa] == [x["n_swapped"] for x in ob]
    for i in range(len(members)):
        for f in (L.FIELD_MASK, L.FIELD_POPS, L.FIELD_UX, L.FIELD_DRHO):
            assert np.array_equal(a.read(i, f), b.read(i, f)), (i, f)
    ta, tb = a.kernel_time(), b.kernel_time()
    assert ta[2] == tb[2]  # the same fluid-cell updates counted
    a.set_step_config(8, persistent=False)  # a fixed shape ends the grouping
    assert a.step_groups() == 1
    ra, rb = a.solve(200), b.solve(200)
    assert [x["dp"] for x in ra] == [x["dp"] for x in rb]
    a.close()
    b.close()


def test_full_candidate_batch_in_groups_matches_alone_and_oracle(ora):
    """The benchmark's batch at full size, in the launch configuration the
    bench times (member groups, tuned shapes): sampled members equal their
    runs alone bit for bit (a handle may pick another kernel; every kernel
    computes the same bits per cell), and one member matches the FP64
    oracle at the FP32 tolerance."""
    cands = I.config_candidates(256)
    members = [dict(cells=c["cells"], tau=c["tau"], u_max=c["u_max"]) for c in cands]
    b = L.Batch(members, residual_every=0)
    rb = b.solve(600)
    assert b.step_groups() > 1
    for i in (0, 37, 101, 200, 255):
        c = cands[i]
        h = L.Lattice(c["cells"], c["tau"], c["u_max"], residual_every=0)
        r = h.solve(600)
        assert r["dp"] == rb[i]["dp"] and np.array_equal(r["m_out"], rb[i]["m_out"]), i
        assert np.array_equal(h.read(L.FIELD_POPS), b.read(i, L.FIELD_POPS)), i
        h.close()
    k = 37
    cells = cands[k]["cells"]
    ny, nx = cells.shape
    s = ora.Solver(ora.make_params(nx, ny, cands[k]["tau"], 1.0, cands[k]["u_max"]), cells, residual_every=0)
    o = s.solve(600)
    ux = b.read(k, L.FIELD_UX).astype(np.float64)
    assert np.abs(ux - s.ux).max() / np.abs(s.ux).max() <= 1e-5
    assert abs(rb[k]["dp"] - o["dp"]) <= 1e-5 * abs(o["dp"])
    b.close()


def test_full_candidate_batch_in_16bit_groups_matches_alone():
    """The 256 candidates with BF16 storage, in the groups of the 16-bit
    budget (two thirds of a third of the L2 of populations: about 4/3 of the
    FP32 groups' cells): at least as many groups as the population bytes
    need, and sampled members equal their runs alone bit for bit."""
    import math
    import torch
    cands = I.config_candidates(256)
    members = [dict(cells=c["cells"], tau=c["tau"], u_max=c["u_max"]) for c in cands]
    b = L.Batch(members, precision=L.BF16_SHIFTED, residual_every=0)
    rb = b.solve(600)
    fluid = sum(int((c["cells"] == 0).sum()) for c in cands)
    l2 = getattr(torch.cuda.get_device_properties(0), "L2_cache_size", 0)
    assert b.step_groups() > 1
    if l2:
        assert b.step_groups() >= math.ceil(9 * 2 * fluid / (l2 / 3.0 * 2.0 / 3.0))
    for i in (0, 101, 255):
        c = cands[i]
        h = L.Lattice(c["cells"], c["tau"], c["u_max"], precision=L.BF16_SHIFTED, residual_every=0)
        r = h.solve(600)
        assert r["dp"] == rb[i]["dp"] and np.array_equal(r["m_out"], rb[i]["m_out"]), i
        assert np.array_equal(h.read(L.FIELD_POPS), b.read(i, L.FIELD_POPS)), i
        h.close()
    b.close()
