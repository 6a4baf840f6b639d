"""Pins of the oracle's optimality-criterion step (Sec. 2.2, Eq. 5-6; Sec. 2.3
steps 3-4): hand-computed scores, brute-force selection on tiny masks, the
fixed fluid volume, the re-initialisation modes."""
import itertools

import numpy as np
import pytest

from paper_1303_0107_gb300 import inputs as I


def _tiny_params(ora, nx=8, ny=8, tau=0.8):
    return ora.make_params(nx, ny, tau, 1.0, 0.01)


def test_hand_computed_scores(ora):
    p = _tiny_params(ora)  # tau 0.8: nu = 0.1, mu = rho0 nu = 0.1
    solid = np.ones((8, 8), np.uint8)
    solid[3:6, 2:6] = 0  # fluid block rows 3..5, cols 2..5
    solid[4, 3] = 1      # one solid cell inside the block
    rho = np.ones((8, 8))
    ux = np.zeros((8, 8))
    uy = np.zeros((8, 8))
    # fluid cell (x=2, y=3): rho 1.2, u = (0.3, 0.4)  -> q = 1/2 * 1.2 * 0.25 = 0.15
    rho[3, 2], ux[3, 2], uy[3, 2] = 1.2, 0.3, 0.4
    # solid cell (x=3, y=4): fluid E (4,4), N (3,5), W (2,4), S (3,3)
    uy[4, 4] = -0.2   # E neighbour: vertical face -> |u_y| = 0.2 -> 0.1*0.2/0.5 = 0.04
    ux[5, 3] = 0.3    # N neighbour: horizontal face -> |u_x| = 0.3 -> 0.06
    ux[4, 2] = 5.0    # W neighbour: its u_x is not tangential to a vertical face
    uy[4, 2] = 0.05   #   ... its u_y is -> 0.01
    ux[3, 3] = -0.1   # S neighbour: |u_x| = 0.1 -> 0.02
    cand, score = ora.scores(p, solid, rho, ux, uy)
    assert cand[3, 2] == 1 and score[3, 2] == pytest.approx(0.15, rel=1e-15)
    assert cand[4, 3] == 2 and score[4, 3] == pytest.approx(0.04 + 0.06 + 0.01 + 0.02, rel=1e-15)
    # solid cell (x=6, y=4): in column nx-2 -> never movable
    assert cand[4, 6] == 0
    # a fluid cell with only fluid 4-neighbours is not interface: (4,4) has solid W (3,4)
    assert cand[4, 4] == 1
    # solid cell (x=4, y=2) below the block: only N neighbour (4,3) fluid; u_x(4,3)=0 -> sigma 0
    assert cand[2, 4] == 2 and score[2, 4] == 0.0


def _brute_force(solid, rho, ux, uy, mu, n_swap):
    ny, nx = solid.shape
    F, S = [], []
    for y in range(1, ny - 1):
        for x in range(2, nx - 2):
            nbs = [(x + 1, y), (x, y + 1), (x - 1, y), (x, y - 1)]
            if solid[y, x] == 0:
                if any(solid[b, a] for a, b in nbs):
                    q = 0.5 * rho[y, x] * (ux[y, x] ** 2 + uy[y, x] ** 2)
                    F.append((q, y * nx + x))
            else:
                terms = []
                for k, (a, b) in enumerate(nbs):
                    if solid[b, a] == 0:
                        ut = uy[b, a] if k in (0, 2) else ux[b, a]
                        terms.append(2.0 * mu * abs(ut))
                if terms:
                    S.append((sum(terms), y * nx + x))
    n = min(n_swap, len(F), len(S))
    F.sort(key=lambda t: (t[0], t[1]))
    S.sort(key=lambda t: (-t[0], t[1]))
    return sorted(i for _, i in F[:n]), sorted(i for _, i in S[:n])


@pytest.mark.parametrize("seed", range(12))
def test_selection_matches_brute_force(ora, seed):
    rng = np.random.default_rng(seed)
    nx, ny = int(rng.integers(6, 9)), int(rng.integers(5, 9))
    p = ora.make_params(nx, ny, 0.8, 1.0, 0.01)
    solid = (rng.random((ny, nx)) < 0.45).astype(np.uint8)
    solid[0, :] = solid[-1, :] = 1
    # quantised velocities: many exact ties exercise the index tie-break
    ux = rng.integers(-2, 3, (ny, nx)) * 0.25
    uy = rng.integers(-2, 3, (ny, nx)) * 0.25
    rho = 1.0 + rng.integers(0, 2, (ny, nx)) * 0.5
    mu = ora.mu_of(p)
    cand, score = ora.scores(p, solid, rho, ux, uy)
    for n_swap in (0, 1, 2, 3, 50):
        fi, si = ora.select(p, cand, score, n_swap)
        bf, bs = _brute_force(solid, rho, ux, uy, mu, n_swap)
        assert list(fi) == bf and list(si) == bs


def test_select_rejects_nan(ora):
    p = _tiny_params(ora)
    solid = np.ones((8, 8), np.uint8)
    solid[3:5, 2:6] = 0
    ux = np.zeros((8, 8))
    ux[3, 3] = np.nan
    cand, score = ora.scores(p, solid, np.ones((8, 8)), ux, np.zeros((8, 8)))
    with pytest.raises(RuntimeError):
        ora.select(p, cand, score, 2)


def test_exchange_keeps_fluid_volume_and_reinitialises(ora):
    cfg = I.config_t_junction()
    p = ora.make_params(cfg["nx"], cfg["ny"], cfg["tau"], 1.0, cfg["u_max"])
    s = ora.Solver(p, cfg["cells"])
    s.solve(400)
    n_fluid = int((s.solid == 0).sum())
    f_before = s.f.copy()
    solid_before = s.solid.copy()
    fi, si = s.pick(5)
    assert len(fi) == 5 and len(si) == 5
    assert all(solid_before.reshape(-1)[fi] == 0) and all(solid_before.reshape(-1)[si] == 1)
    count = s.exchange(fi, si)
    assert count == n_fluid == int((s.solid == 0).sum())
    cx, cy, opp, w, _ = ora.lattice()
    ff = s.f.reshape(9, -1)
    for c in si:  # new fluid cells at the rest equilibrium of rho0
        assert np.array_equal(ff[:, c], w * 1.0)
    for c in fi:  # new solid cells hold no state
        assert np.all(ff[:, c] == 0.0)
    keep = (solid_before.reshape(-1) == 0) & (s.solid.reshape(-1) == 0)
    assert np.array_equal(ff[:, keep], f_before.reshape(9, -1)[:, keep])


def test_cold_reinit_resets_every_fluid_cell(ora):
    cfg = I.config_t_junction()
    p = ora.make_params(cfg["nx"], cfg["ny"], cfg["tau"], 1.0, cfg["u_max"])
    s = ora.Solver(p, cfg["cells"], reinit=ora.REINIT_COLD)
    s.solve(200)
    fi, si = s.pick(3)
    s.exchange(fi, si)
    cx, cy, opp, w, _ = ora.lattice()
    ff = s.f.reshape(9, -1)
    fluid = s.solid.reshape(-1) == 0
    assert np.array_equal(ff[:, fluid], np.repeat((w * 1.0)[:, None], fluid.sum(), axis=1))


def test_ports_and_frame_never_move(ora):
    cfg = I.config_t_junction()
    p = ora.make_params(cfg["nx"], cfg["ny"], cfg["tau"], 1.0, cfg["u_max"])
    s = ora.Solver(p, cfg["cells"])
    s.solve(200)
    for _ in range(3):
        fi, si = s.pick(40)
        for idx in itertools.chain(fi, si):
            y, x = divmod(int(idx), p.nx)
            assert 2 <= x <= p.nx - 3 and 1 <= y <= p.ny - 2
        s.exchange(fi, si)
        s.solve(50)


@pytest.mark.slow
def test_t_junction_optimisation_lowers_pressure_drop(ora):
    """Sec. 2.3 reports that the optimisation turns a T into a Y with a lower
    pressure drop; the size of the drop is not comparable (geometry unknown),
    only its direction.  Ten exchanges of two cells on the 128 x 64 T-junction,
    each followed by 2000 steps, against the unchanged T run for the same
    22000 steps (the first 2000-step solve is still far from steady)."""
    cfg = I.config_t_junction()
    p = ora.make_params(cfg["nx"], cfg["ny"], cfg["tau"], 1.0, cfg["u_max"])
    total = cfg["steps"] * (cfg["n_iter"] + 1)
    dp_unchanged = ora.Solver(p, cfg["cells"]).solve(total)["dp"]
    s = ora.Solver(p, cfg["cells"])
    s.solve(cfg["steps"])
    n0 = int((s.solid == 0).sum())
    for _ in range(cfg["n_iter"]):
        out = s.optimize_step(2, cfg["steps"])
        assert out["fluid_count"] == n0
    assert out["dp"] < 0.95 * dp_unchanged


# ---- the outer loop's decisions (stopping test, n_swap adaptation, best) ----

def _fake(seq):
    it = iter(seq)
    calls = []

    def solve():
        return next(it)

    def step(ns):
        calls.append(ns)
        return next(it)
    return solve, step, calls


def test_run_plan_without_tolerance_runs_every_iteration(ora):
    seq = [5.0, 4.0, 4.5, 3.0, 3.0, 3.5]
    solve, step, calls = _fake(seq)
    out = ora.run_plan(solve, step, n_swap=8, max_iter=5)
    assert out["history"] == seq and out["iterations"] == 5 and not out["stopped"]
    assert out["best_iter"] == 3 and out["dp_best"] == 3.0  # earliest of the two equal minima
    assert calls == [8] * 5 and out["n_swap_final"] == 8


def test_run_plan_stops_after_patience_calm_iterations(ora):
    # relative changes: 0.1, 1e-4, 2e-4, 5e-2, 1e-4, 1e-4, 1e-4 (stop here with patience 3)
    seq = [1.0, 0.9, 0.90009, 0.90027, 0.95, 0.950095, 0.95019, 0.950285, 0.5]
    solve, step, calls = _fake(seq)
    out = ora.run_plan(solve, step, n_swap=4, max_iter=8, tol=1e-3, patience=3)
    assert out["stopped"] and out["iterations"] == 7 and len(calls) == 7
    assert out["best_iter"] == 1
    solve, step, calls = _fake(seq)
    out = ora.run_plan(solve, step, n_swap=4, max_iter=8, tol=1e-3, patience=4)
    assert not out["stopped"] and out["iterations"] == 8 and out["best_iter"] == 8


def test_run_plan_halves_n_swap_after_a_rise(ora):
    seq = [10.0, 9.0, 9.5, 8.0, 8.5, 8.6, 8.7, 7.0]
    solve, step, calls = _fake(seq)
    out = ora.run_plan(solve, step, n_swap=10, max_iter=7, adapt=True)
    # rises after iterations 2, 4, 5, 6: 10 -> 5 -> 2 -> 1 -> 1
    assert calls == [10, 10, 5, 5, 2, 1, 1]
    assert out["n_swap_final"] == 1 and out["best_iter"] == 7


def test_optimize_run_keep_best_restores_the_best_state(ora):
    cfg = I.config_t_junction()
    p = ora.make_params(cfg["nx"], cfg["ny"], cfg["tau"], 1.0, cfg["u_max"])
    ref = ora.Solver(p, cfg["cells"], residual_every=0)
    states = [None]
    dps = [ref.solve(200)["dp"]]
    states[0] = ref.solid.copy()
    for _ in range(4):
        dps.append(ref.optimize_step(3, 200)["dp"])
        states.append(ref.solid.copy())
    s = ora.Solver(p, cfg["cells"], residual_every=0)
    out = s.optimize_run(200, 4, 3, keep_best=True)
    assert out["history"] == dps
    assert out["best_iter"] == int(np.argmin(dps))
    assert np.array_equal(s.solid, states[out["best_iter"]])
    assert int((s.solid == 0).sum()) == int((cfg["cells"] == 0).sum())


# ---- connectivity guard (simple cells only may turn solid) ----

def _components(fluid):
    """Number of 4-connected components of a boolean array (brute force)."""
    seen = np.zeros_like(fluid, dtype=bool)
    ny, nx = fluid.shape
    n = 0
    for y0 in range(ny):
        for x0 in range(nx):
            if not fluid[y0, x0] or seen[y0, x0]:
                continue
            n += 1
            stack = [(y0, x0)]
            seen[y0, x0] = True
            while stack:
                y, x = stack.pop()
                for dy, dx in ((0, 1), (1, 0), (0, -1), (-1, 0)):
                    yy, xx = y + dy, x + dx
                    if 0 <= yy < ny and 0 <= xx < nx and fluid[yy, xx] and not seen[yy, xx]:
                        seen[yy, xx] = True
                        stack.append((yy, xx))
    return n


def _solid_components8(solid):
    """8-connected components of the solid cells (brute force)."""
    seen = np.zeros_like(solid, dtype=bool)
    ny, nx = solid.shape
    n = 0
    for y0 in range(ny):
        for x0 in range(nx):
            if not solid[y0, x0] or seen[y0, x0]:
                continue
            n += 1
            stack = [(y0, x0)]
            seen[y0, x0] = True
            while stack:
                y, x = stack.pop()
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        yy, xx = y + dy, x + dx
                        if 0 <= yy < ny and 0 <= xx < nx and solid[yy, xx] and not seen[yy, xx]:
                            seen[yy, xx] = True
                            stack.append((yy, xx))
    return n


def test_simple_cells_are_exactly_those_whose_removal_keeps_the_local_topology(ora):
    """Brute force over every 3 x 3 neighbourhood: the centre is simple iff
    removing it leaves one 4-connected fluid part among its fluid 4-neighbour
    connections and merges no solid parts -- checked as: the fluid cells of
    the 3 x 3 block that were 4-connected to the centre stay in one
    4-component, and the solid 8-components of the block do not change."""
    p = ora.make_params(3, 3, 0.8, guard=True)
    for code in range(256):
        ring = [(code >> k) & 1 for k in range(8)]  # fluid flags E, NE, N, NW, W, SW, S, SE
        DX = [1, 1, 0, -1, -1, -1, 0, 1]
        DY = [0, 1, 1, 1, 0, -1, -1, -1]
        fluid = np.zeros((3, 3), bool)
        fluid[1, 1] = True
        for k in range(8):
            fluid[1 + DY[k], 1 + DX[k]] = bool(ring[k])
        solid = (~fluid).astype(np.uint8)
        got = ora.simple(p, solid, 1, 1)
        after = fluid.copy()
        after[1, 1] = False
        # fluid 4-neighbours of the centre must stay 4-connected to one another (within the block)
        nb4 = [(1 + DY[k], 1 + DX[k]) for k in (0, 2, 4, 6) if ring[k]]
        lab = np.zeros((3, 3), int)
        comp = 0
        for (y, x) in nb4:
            if lab[y, x]:
                continue
            comp += 1
            stack = [(y, x)]
            lab[y, x] = comp
            while stack:
                cy, cx = stack.pop()
                for dy, dx in ((0, 1), (1, 0), (0, -1), (-1, 0)):
                    yy, xx = cy + dy, cx + dx
                    if 0 <= yy < 3 and 0 <= xx < 3 and after[yy, xx] and not lab[yy, xx]:
                        lab[yy, xx] = comp
                        stack.append((yy, xx))
        keeps_fluid = comp == 1
        # the removed cell joins the solid: it must touch exactly one 8-component of the block's solid
        sol = ~fluid
        sol[1, 1] = False
        n_before = _solid_components8(sol)
        sol2 = sol.copy()
        sol2[1, 1] = True
        keeps_solid = n_before >= 1 and _solid_components8(sol2) == n_before
        assert got == int(keeps_fluid and keeps_solid), (code, ring)


def test_guarded_choice_never_cuts_a_one_cell_neck(ora):
    """A channel pinched to a neck one to three cells wide: every fluid cell
    the guard lets turn solid leaves the number of fluid components as it
    was."""
    rng = np.random.default_rng(3)
    for trial in range(20):
        nx, ny = 12, 9
        solid = np.ones((ny, nx), np.uint8)
        solid[2:7, :] = 0
        # a random wall bump leaves a neck one to three cells wide
        xb = int(rng.integers(4, nx - 4))
        w = int(rng.integers(1, 4))
        solid[2:7 - w, xb] = 1
        p = ora.make_params(nx, ny, 0.8, u_max=0.02, guard=True)
        rho = np.ones((ny, nx))
        ux = rng.random((ny, nx)) * (solid == 0)
        uy = rng.random((ny, nx)) * (solid == 0) * 0.1
        cand, score = ora.scores(p, solid, rho, ux, uy)
        for c in np.flatnonzero(cand == 1):
            y, x = divmod(int(c), nx)
            after = solid.copy()
            after[y, x] = 1
            assert _components(after == 0) == _components(solid == 0), (trial, x, y)
