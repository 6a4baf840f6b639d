"""The C-ABI's geometry rules are host logic, checked before any device
call: on random cell maps (valid distributors and mutated ones) the
libraries' answers (LBM_ERR_GEOMETRY or not) must equal the oracles' rules
plus the rules the oracles leave to the caller (an inlet and an outlet cell,
at most LBM_MAX_OUTLETS outlet runs or regions), computed here by brute
force.  Runs without a GPU: a valid map then fails at the first device call
(LBM_ERR_CUDA), which is not a geometry answer."""
import ctypes

import numpy as np
import pytest

import oracle as ora2
from oracle import lbm3d as o3
from paper_1303_0107_gb300 import inputs as I
from paper_1303_0107_gb300 import lib, lib3d

GEOMETRY = 2


def _status2(cells, mirror=False):
    L = lib.load_library()
    ny, nx = cells.shape
    p = lib.make_params(nx, ny, 0.8, 0.05, mirror=mirror)
    h = ctypes.c_void_p()
    st = L.lbm_create_geometry(ctypes.byref(p), np.ascontiguousarray(cells, np.uint8).ctypes.data, None,
                               ctypes.byref(h))
    if h.value:
        L.lbm_destroy(h)
    return st


def _status3(cells, mirror=False):
    L = lib3d._lib()
    nz, ny, nx = cells.shape
    p = lib3d.make_params3(nx, ny, nz, 0.8, 0.05, mirror=mirror)
    h = ctypes.c_void_p()
    st = L.lbm3d_create(ctypes.byref(p), np.ascontiguousarray(cells, np.uint8).ctypes.data, None, ctypes.byref(h))
    if h.value:
        L.lbm3d_destroy(h)
    return st


def _runs(col):
    """Number of runs of fluid cells (0) in a 1D column."""
    f = (np.asarray(col) == 0).astype(int)
    return int(((f[1:] == 1) & (f[:-1] == 0)).sum() + f[0])


def _mutations2(base, rng):
    ny, nx = base.shape
    out = [base.copy()]
    for _ in range(12):
        c = base.copy()
        kind = rng.integers(0, 6)
        if kind == 0:    # a hole in the frame
            c[rng.choice([0, ny - 1]), rng.integers(0, nx)] = 0
        elif kind == 1:  # an inlet cell with a wall behind it
            ys = np.flatnonzero(c[:, 0] == 0)
            if len(ys):
                c[rng.choice(ys), 1] = 1
        elif kind == 2:  # an outlet cell with a wall before it
            ys = np.flatnonzero(c[:, -1] == 0)
            if len(ys):
                c[rng.choice(ys), -2] = 1
        elif kind == 3:  # no inlet at all
            c[:, 0] = 1
        elif kind == 4:  # no outlet at all
            c[:, -1] = 1
        else:            # random interior flips (still valid)
            ys, xs = rng.integers(1, ny - 1, 20), rng.integers(2, nx - 2, 20)
            c[ys, xs] ^= 1
        out.append(c)
    return out


def test_2d_geometry_answers_match_the_rules():
    rng = np.random.default_rng(4)
    n_bad = 0
    for cand in I.config_candidates(6):
        for c in _mutations2(cand["cells"], rng):
            ny, nx = c.shape
            rule_bad = ora2.check_geometry(ora2.make_params(nx, ny, 0.8), c) != 0
            rule_bad |= (c[:, 0] == 0).sum() == 0 or (c[:, -1] == 0).sum() == 0
            rule_bad |= _runs(c[:, -1]) > lib.MAX_OUTLETS
            st = _status2(c)
            assert (st == GEOMETRY) == rule_bad, (st, rule_bad)
            n_bad += rule_bad
    assert n_bad > 10  # the mutations do break the rules


def test_2d_too_many_outlet_runs_and_the_mirror_row():
    nx, ny = 64, 2 * (lib.MAX_OUTLETS + 1) + 1
    c = np.ones((ny, nx), np.uint8)
    c[1:-1, :] = 0
    c[2:-1:2, -8:] = 1  # 65 outlet runs separated by single walls
    assert _runs(c[:, -1]) == lib.MAX_OUTLETS + 1
    assert ora2.check_geometry(ora2.make_params(nx, ny, 0.8), c) == 0
    assert _status2(c) == GEOMETRY
    half = np.ones((12, 40), np.uint8)
    half[0:6, :] = 0  # row 0 fluid: valid next to a symmetry plane only
    assert _status2(half) == GEOMETRY and _status2(half, mirror=True) != GEOMETRY


def _mutations3(base, rng):
    nz, ny, nx = base.shape
    out = [base.copy()]
    for _ in range(10):
        c = base.copy()
        kind = rng.integers(0, 5)
        if kind == 0:
            c[rng.choice([0, nz - 1]), rng.integers(0, ny), rng.integers(0, nx)] = 0
        elif kind == 1:
            c[rng.integers(0, nz), rng.choice([0, ny - 1]), rng.integers(0, nx)] = 0
        elif kind == 2:
            zs, ys = np.nonzero(c[:, :, 0] == 0)
            if len(zs):
                k = rng.integers(0, len(zs))
                c[zs[k], ys[k], 1] = 1
        elif kind == 3:
            c[:, :, -1] = 1
        else:
            zs, ys, xs = rng.integers(1, nz - 1, 30), rng.integers(1, ny - 1, 30), rng.integers(2, nx - 2, 30)
            c[zs, ys, xs] ^= 1
        out.append(c)
    return out


def test_3d_geometry_answers_match_the_rules():
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(5)
    n_bad = 0
    for base in (I.config_tree3d_small()["cells"], I.random_blobs3d(40, 10, 9, seed=1, density=0.1)):
        for c in _mutations3(base, rng):
            nz, ny, nx = c.shape
            rule_bad = o3.check_geometry3(o3.make_params3(nx, ny, nz, 0.8), c) != 0
            rule_bad |= ndi.label(c[:, :, -1] == 0)[1] > lib.MAX_OUTLETS
            st = _status3(c)
            assert (st == GEOMETRY) == rule_bad, (st, rule_bad)
            n_bad += rule_bad
    assert n_bad > 5
    half = np.ascontiguousarray(I.config_tree3d_small()["cells"][:, 17:, :])
    assert _status3(half) == GEOMETRY and _status3(half, mirror=1) != GEOMETRY
    quarter = np.ascontiguousarray(I.config_tree3d_small()["cells"][17:, 17:, :])
    assert _status3(quarter, mirror=1) == GEOMETRY and _status3(quarter, mirror=2) == GEOMETRY
    assert _status3(quarter, mirror=3) != GEOMETRY
