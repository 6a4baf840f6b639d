"""The request loop (lbm_server_*): continuous batching with admission by
device footprint.

The key property: a request's results are the same served in a mix of other
requests -- admitted and retired around it at tick boundaries, exchanges of
other requests interleaved -- as computed alone on a handle of its own.  The
kernels compute each member from its own data in an order fixed by the
member, so equality is expected bit for bit; the stated gate is a relative
pressure-drop difference of at most 1e-4.
"""
import time

import numpy as np
import pytest

import paper_1303_0107_gb300 as L
from paper_1303_0107_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DP_GATE = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load_library()


def _requests(n, seed0, n_steps=400, max_nx=512):
    """Served-request geometries (small sizes so the alone runs stay short):
    every third request optimises for 3 iterations, the others solve."""
    out = []
    s = seed0
    while len(out) < n:
        r = I.config_served_request(s)
        s += 1
        if r["nx"] > max_nx:
            continue
        k = len(out)
        opt = k % 3 == 1
        fluid = int((r["cells"] == 0).sum())
        out.append(dict(tag=1000 + k, cells=r["cells"], tau=r["tau"], u_max=r["u_max"], n_steps=n_steps,
                        n_iter=3 if opt else 0, n_swap=max(1, fluid // 500) if opt else 0,
                        steps=n_steps + (k % 4) * 100))
    for q in out:  # uneven solve lengths so that ticks are cut at many points
        q["n_steps"] = q.pop("steps")
    return out


def _alone(q, precision):
    h = L.Lattice(q["cells"], q["tau"], q["u_max"], precision=precision, residual_every=0)
    first = h.solve(q["n_steps"])
    last, swapped = first, 0
    for _ in range(q["n_iter"]):
        last = h.optimize_step(q["n_swap"], q["n_steps"])
        swapped += last["n_swapped"]
    fields = dict(mask=h.read(L.FIELD_MASK), drho=h.read(L.FIELD_DRHO), ux=h.read(L.FIELD_UX),
                  uy=h.read(L.FIELD_UY))
    h.close()
    return first, last, swapped, fields


def _serve(reqs, precision, stagger_s=0.002, **cfg):
    srv = L.Server(precision=precision, **cfg)
    for q in reqs:
        srv.submit(q["tag"], q["cells"], q["tau"], q["u_max"], q["n_steps"], n_iter=q["n_iter"],
                   n_swap=q["n_swap"], keep_fields=True)
        time.sleep(stagger_s)  # arrivals while others are on the device
    srv.wait_idle(300)
    done = {}
    while True:
        got = srv.poll(64)
        if not got:
            break
        for d in got:
            done[d["tag"]] = d
    stats = srv.stats()
    srv.close()
    return done, stats


@pytest.mark.parametrize("precision", [L.F32, L.BF16_SHIFTED])
def test_served_results_equal_alone(precision):
    reqs = _requests(20, 300)
    done, stats = _serve(reqs, precision, max_tick_steps=200)
    assert len(done) == len(reqs)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["peak_active"] >= 2, "requests never overlapped on the device"
    worst = 0.0
    for q in reqs:
        d = done[q["tag"]]
        assert d["status"] == 0, d
        first, last, swapped, f = _alone(q, precision)
        rel = abs(d["last"]["dp"] - last["dp"]) / abs(last["dp"])
        worst = max(worst, rel)
        assert rel <= DP_GATE
        # expected bit for bit
        assert d["dp_first"] == first["dp"], q["tag"]
        assert d["last"]["dp"] == last["dp"], q["tag"]
        assert np.array_equal(d["last"]["m_out"], last["m_out"])
        assert d["n_swapped"] == swapped
        assert d["last"]["fluid_cells"] == int((q["cells"] == 0).sum())
        for k in ("mask", "drho", "ux", "uy"):
            assert np.array_equal(d["fields"][k], f[k]), (q["tag"], k)
        assert d["fluid_updates"] == last["fluid_cells"] * q["n_steps"] * (1 + q["n_iter"])
        assert d["t_submit"] <= d["t_admit"] <= d["t_done"]
    print(f"worst served-vs-alone relative dp difference: {worst:.3g}")


def test_admission_respects_the_budget():
    reqs = _requests(8, 500, n_steps=200)
    fps = [L.Server.footprint(q["cells"].shape[1], q["cells"].shape[0], q["n_iter"]) for q in reqs]
    budget = sorted(fps)[-1] + sorted(fps)[-2]  # room for about two requests at a time
    done, stats = _serve(reqs, L.F32, stagger_s=0.0, hbm_budget_bytes=budget, max_tick_steps=100)
    assert stats["completed"] == len(reqs)
    assert stats["budget_bytes"] == budget
    assert 0 < stats["peak_resident_bytes"] <= budget
    assert stats["peak_active"] < len(reqs)  # the budget made later requests wait
    for q in reqs[:3]:
        _, last, _, f = _alone(q, L.F32)
        assert done[q["tag"]]["last"]["dp"] == last["dp"]


def test_single_slot_is_first_come_first_served():
    reqs = _requests(4, 700, n_steps=200)
    done, stats = _serve(reqs, L.F32, stagger_s=0.0, max_active=1)
    assert stats["peak_active"] == 1
    order = sorted(done.values(), key=lambda d: d["t_done"])
    assert [d["tag"] for d in order] == [q["tag"] for q in reqs]


def test_submit_errors():
    srv = L.Server(precision=L.F32, hbm_budget_bytes=1 << 20)
    t = I.config_t_junction()
    with pytest.raises(L.LbmError) as e:  # odd step count
        srv.submit(1, t["cells"], t["tau"], t["u_max"], 301)
    assert e.value.status == 1
    big = I.config_tree_2048()
    with pytest.raises(L.LbmError) as e:  # never fits the 1 MiB budget
        srv.submit(2, big["cells"], big["tau"], big["u_max"], 100)
    assert e.value.status == 1
    bad = t["cells"].copy()
    bad[0, :] = 0  # frame row open
    with pytest.raises(L.LbmError) as e:
        srv.submit(3, bad, t["tau"], t["u_max"], 100)
    assert e.value.status == 2
    srv.close()
    srv = L.Server(precision=L.BF16_SHIFTED)
    with pytest.raises(L.LbmError):  # precision differs from the server's
        r = L.lib.Request()
        r.params = L.Server.params_for(t["cells"], t["tau"], t["u_max"], precision=L.F32)
        r.cell_types = np.ascontiguousarray(t["cells"]).ctypes.data
        r.n_steps = 100
        L.lib._check(L.load_library().lbm_server_submit(srv._s, r), "lbm_server_submit")
    assert srv.stats()["submitted"] == 0
    srv.close()


def test_cancel_queued_and_resident_requests():
    reqs = _requests(5, 900, n_steps=400)
    reqs[0]["n_steps"] = 400000  # long enough to be resident when it is withdrawn
    srv = L.Server(precision=L.F32, max_active=1, max_tick_steps=200)
    for q in reqs:
        srv.submit(q["tag"], q["cells"], q["tau"], q["u_max"], q["n_steps"], n_iter=q["n_iter"], n_swap=q["n_swap"])
    srv.cancel(reqs[3]["tag"])  # queued behind the long one
    t0 = time.time()
    while srv.stats()["admitted"] < 1 and time.time() - t0 < 30:
        time.sleep(0.005)
    srv.cancel(reqs[0]["tag"])  # resident: withdrawn at the next tick boundary
    with pytest.raises(L.LbmError):
        srv.cancel(123456789)
    srv.wait_idle(300)
    done = {d["tag"]: d for d in srv.poll(64)}
    srv.close()
    assert len(done) == 5
    assert done[reqs[3]["tag"]]["status"] == 8 and done[reqs[0]["tag"]]["status"] == 8
    assert done[reqs[0]["tag"]]["fluid_updates"] < int((reqs[0]["cells"] == 0).sum()) * 400000
    for k in (1, 2, 4):
        assert done[reqs[k]["tag"]]["status"] == 0
        _, last, _, _ = _alone(reqs[k], L.F32)
        assert done[reqs[k]["tag"]]["last"]["dp"] == last["dp"]


def test_failed_allocation_fails_only_its_request():
    reqs = _requests(3, 950, n_steps=200)
    srv = L.Server(precision=L.F32, max_active=4, max_tick_steps=100)
    L.lib.debug_fail_alloc(0)  # the next device allocation: the first request's storage
    for q in reqs:
        srv.submit(q["tag"], q["cells"], q["tau"], q["u_max"], q["n_steps"])
    srv.wait_idle(300)
    L.lib.debug_fail_alloc(-1)
    done = {d["tag"]: d for d in srv.poll(64)}
    st = srv.stats()
    srv.close()
    assert done[reqs[0]["tag"]]["status"] == 3  # LBM_ERR_OOM
    assert [done[q["tag"]]["status"] for q in reqs[1:]] == [0, 0]
    assert st["failed"] == 1 and st["resident_bytes"] == 0


def test_a_diverging_request_fails_alone():
    """A request that blows up (BGK at tau = 0.51 past a block: non-finite
    density within 4000 steps) is reported LBM_ERR_DIVERGED; the requests
    stepped in the same launches beside it finish as they would alone, bit
    for bit."""
    cells = np.ones((60, 200), np.uint8)
    cells[1:-1, :] = 0
    cells[22:38, 50:56] = 1
    reqs = _requests(3, 700, n_steps=300)
    srv = L.Server(precision=L.F32, max_active=8, max_tick_steps=500)
    srv.submit(99, cells, 0.51, 0.05, 4000)
    for q in reqs:
        srv.submit(q["tag"], q["cells"], q["tau"], q["u_max"], q["n_steps"], n_iter=q["n_iter"],
                   n_swap=q["n_swap"])
    srv.wait_idle(300)
    done = {d["tag"]: d for d in srv.poll(64)}
    st = srv.stats()
    srv.close()
    assert done[99]["status"] == 5  # LBM_ERR_DIVERGED
    assert st["failed"] == 1 and st["completed"] == len(reqs)
    for q in reqs:
        d = done[q["tag"]]
        assert d["status"] == 0, d
        first, last, swapped, _ = _alone(q, L.F32)
        assert d["dp_first"] == first["dp"] and d["last"]["dp"] == last["dp"], q["tag"]
        assert d["n_swapped"] == swapped
