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
