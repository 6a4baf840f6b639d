"""lbm_optimize: the whole loop of Sec. 2.3 in one call, with the stopping
test, n_swap adaptation and best-state keeping of lbm_opt_plan.

The loop must take exactly the decisions the oracle's run_plan takes on the
same pressure-drop sequence, and compute exactly what the same sequence of
lbm_solve / lbm_optimize_step calls computes (bit for bit).
"""
import numpy as np
import pytest

import oracle as ora
import paper_1303_0107_gb300 as L
from paper_1303_0107_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load_library()


def _reference(cfg, n_steps, max_iter, n_swap, **plan):
    """The same plan driven from Python through the per-step entry points."""
    h = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"], residual_every=0)
    masks, ux = [], []

    def solve():
        dp = h.solve(n_steps)["dp"]
        masks.append(h.read(L.FIELD_MASK))
        ux.append(h.read(L.FIELD_UX))
        return dp

    def step(ns):
        dp = h.optimize_step(ns, n_steps)["dp"]
        masks.append(h.read(L.FIELD_MASK))
        ux.append(h.read(L.FIELD_UX))
        return dp

    out = ora.run_plan(solve, step, n_swap, max_iter, **plan)
    h.close()
    return out, masks, ux


@pytest.mark.parametrize("plan", [dict(), dict(adapt=True), dict(tol=2e-2, patience=2, adapt=True)])
def test_loop_equals_per_step_calls_and_oracle_decisions(plan):
    cfg = I.config_t_junction()
    ref, masks, ux = _reference(cfg, 400, 8, 6, **plan)
    h = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"], residual_every=0)
    got = h.optimize(400, 8, 6, keep_best=False, **plan)
    assert list(got["history"]) == ref["history"]
    assert got["iterations"] == ref["iterations"] and bool(got["stopped"]) == ref["stopped"]
    assert got["best_iter"] == ref["best_iter"] and got["dp_best"] == ref["dp_best"]
    assert got["n_swap_final"] == ref["n_swap_final"]
    assert got["dp_first"] == ref["history"][0] and got["dp_last"] == ref["history"][-1]
    assert np.array_equal(h.read(L.FIELD_MASK), masks[-1])
    h.close()


def test_keep_best_ends_in_the_best_state():
    cfg = I.config_t_junction()
    ref, masks, ux = _reference(cfg, 400, 6, 8)
    h = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"], residual_every=0)
    got = h.optimize(400, 6, 8, keep_best=True)
    b = got["best_iter"]
    assert b == ref["best_iter"] and list(got["history"]) == ref["history"]
    assert np.array_equal(h.read(L.FIELD_MASK), masks[b])
    assert np.array_equal(h.read(L.FIELD_UX), ux[b])
    # the restored state continues like the best iteration's state would
    r = h.solve(2)
    assert r["fluid_cells"] == int((cfg["cells"] == 0).sum())
    h.close()


def test_extremum_test_stops_the_loop():
    cfg = I.config_t_junction()
    h = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"], residual_every=0)
    got = h.optimize(400, 10, 2, tol=1.0, patience=2)  # every change is calm at tol = 1
    assert got["stopped"] == 1 and got["iterations"] == 2 and len(got["history"]) == 3
    h.close()


def test_plan_errors():
    cfg = I.config_t_junction()
    h = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"], residual_every=0)
    for kw in (dict(n_steps=401, max_iter=2, n_swap=2), dict(n_steps=400, max_iter=-1, n_swap=2),
               dict(n_steps=400, max_iter=2, n_swap=0), dict(n_steps=400, max_iter=2, n_swap=2, patience=0)):
        with pytest.raises(L.LbmError) as e:
            h.optimize(**kw)
        assert e.value.status == 1
    h.close()
