"""Properties of the seeded synthetic inputs (no method arithmetic here)."""
import numpy as np

from paper_1303_0107_gb300 import inputs as I


def _ports_ok(cells):
    ny, nx = cells.shape
    assert cells[0].all() and cells[-1].all()
    for y in range(ny):
        if cells[y, 0] == 0:
            assert cells[y, 1] == 0
        if cells[y, -1] == 0:
            assert cells[y, -2] == 0


def _runs(col):
    runs, y = [], 0
    while y < len(col):
        if col[y] == 0:
            y0 = y
            while y < len(col) and col[y] == 0:
                y += 1
            runs.append((y0, y - y0))
        else:
            y += 1
    return runs


def test_t_junction_layout():
    c = I.config_t_junction()
    cells = c["cells"]
    assert cells.shape == (64, 128) and cells.dtype == np.uint8
    _ports_ok(cells)
    assert _runs(cells[:, 0]) == [(28, 8)]
    assert [w for _, w in _runs(cells[:, -1])] == [4, 4]
    assert 1000 < int((cells == 0).sum()) < 1300


def test_tree_2048_layout():
    c = I.config_tree_2048()
    cells = c["cells"]
    _ports_ok(cells)
    assert [w for _, w in _runs(cells[:, 0])] == [64]
    outs = _runs(cells[:, -1])
    assert len(outs) == 16 and all(w == 4 for _, w in outs)
    # outlet centres uniformly spaced ny / 2^G apart
    centres = [y + w / 2 for y, w in outs]
    assert np.allclose(np.diff(centres), 1024 / 16)
    frac = (cells == 0).mean()
    assert 0.05 < frac < 0.12


def test_unjittered_tree_is_mirror_symmetric():
    for G, W in [(1, [8, 4]), (2, [8, 4, 4]), (4, [64, 32, 16, 8, 4])]:
        ny = 64 if G < 4 else 1024
        nx = 2 * ny
        cells = I.tree(nx, ny, G, W[0], widths=W, jitter=0)
        assert np.array_equal(cells, cells[::-1])


def test_seeded_determinism_and_jitter():
    a = I.tree(512, 256, 3, 32, jitter=2, seed=5)
    b = I.tree(512, 256, 3, 32, jitter=2, seed=5)
    c = I.tree(512, 256, 3, 32, jitter=2, seed=6)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert I.splitmix64(0, 0) == I.splitmix64(0, 0)


def test_candidates_and_requests_are_valid():
    for c in I.config_candidates(16):
        _ports_ok(c["cells"])
        assert 256 <= c["nx"] <= 1024 and c["nx"] % 32 == 0 and c["ny"] == c["nx"] // 2
        assert len(_runs(c["cells"][:, -1])) == 2 ** c["generations"]
    for s in range(16):
        r = I.config_served_request(s)
        _ports_ok(r["cells"])
        assert 128 <= r["nx"] <= 2048


def test_poisson_arrivals_rate():
    t = I.poisson_arrivals(200.0, 30.0, seed=1)
    assert 5400 < len(t) < 6600 and all(np.diff(t) > 0)


def test_collector_replica_geometry(ora):
    """The paper's half-domain collector (Sec. 3.3): 8 inlets of 11 cells,
    one 52-cell outlet against the symmetry plane, Re = 22."""
    c = I.config_collector()
    cells = c["cells"]
    assert cells.shape == (180, 360)
    col0 = np.flatnonzero(cells[:, 0] == 0)
    runs = np.split(col0, np.flatnonzero(np.diff(col0) > 1) + 1)
    assert [len(r) for r in runs] == [11] * 8
    out = np.flatnonzero(cells[:, -1] == 0)
    assert out[0] == 0 and len(out) == 52 and np.all(np.diff(out) == 1)
    assert cells[-1].all() and not cells[0].all()
    p = ora.make_params(360, 180, c["tau"], 1.0, c["u_max"], outlet_rule=c["outlet"], mirror=True)
    assert ora.check_geometry(p, cells) == 0
    nu = (c["tau"] - 0.5) / 3
    assert abs(11 * (2 / 3) * c["u_max"] / nu - 22) < 1e-9
