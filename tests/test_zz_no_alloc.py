"""The exchange selection for callers that cannot allocate device memory.

Code that runs inside an application whose memory pool owns the GPU, or a
loop that must not risk the device-wide synchronisation of cudaMalloc and
cudaFree, cannot use the handle-based entry points (creating a handle
allocates).  lbm_select_swaps_noalloc takes only caller-owned device buffers
and keeps its intermediate data in a static device array.  Here it is called
through the C ABI twice in a row, on two lattices of different shapes (so
anything left over in the shared array from the first call would show), and
its picks must equal those of lbm_select_swaps and of the FP64 oracle's
selection on the same fields bit for bit.  The edge cases: more cells asked
for than there are candidates (n is clamped), a field holding a NaN (n_out
= -1), and n_swap = 0 with no output buffers (n_out = 0).  This file is
named to be collected last.
"""

import numpy as np
import pytest

import paper_1303_0107_gb300 as L
from paper_1303_0107_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MAX_CELLS = 262144  # LBM_NOALLOC_MAX_CELLS in include/lbm.h


def _fields(shape, seed, ties):
    rng = np.random.default_rng(seed)
    drho = (0.01 * rng.standard_normal(shape)).astype(np.float32)
    ux = (0.05 * rng.standard_normal(shape)).astype(np.float32)
    uy = (0.05 * rng.standard_normal(shape)).astype(np.float32)
    if ties:
        ux = (np.round(ux * 40) / 40).astype(np.float32)
        uy = (np.round(uy * 40) / 40).astype(np.float32)
        drho[:] = 0
    return drho, ux, uy


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _noalloc(lib, torch, cells, tau, drho, ux, uy, n_swap, with_outputs=True):
    """One call through the C ABI on device copies; returns (status, n_out, fluid picks, solid picks)."""
    ny, nx = cells.shape
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (cells, drho, ux, uy)]
    cap = max(n_swap, 1)
    out_f = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    out_s = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    n_dev = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    st = lib.lbm_select_swaps_noalloc(nx, ny, tau, 1.0, *[t.data_ptr() for t in dev], n_swap,
                                      out_f.data_ptr() if with_outputs else None,
                                      out_s.data_ptr() if with_outputs else None, n_dev.data_ptr(),
                                      stream.cuda_stream)
    torch.cuda.synchronize()
    n = int(n_dev.item())
    k = max(n, 0)
    return st, n, out_f[:k].cpu().numpy(), out_s[:k].cpu().numpy()


def _oracle_pick(ora, cells, tau, drho, ux, uy, n_swap):
    ny, nx = cells.shape
    p = ora.make_params(nx, ny, tau, 1.0)
    rho = 1.0 + drho.astype(np.float64)
    cand, score = ora.scores(p, cells, rho, ux.astype(np.float64), uy.astype(np.float64))
    return ora.select(p, cand, score, n_swap)


def test_noalloc_selection_equals_handle_and_oracle_twice(ora):
    torch = _torch()
    lib = L.load_library()
    t_junction = I.config_t_junction()
    cases = [(t_junction["cells"], t_junction["tau"], 7, 0, False),
             (I.random_blobs(100, 40, 5, density=0.3), 0.7, 25, 1, True)]
    for cells, tau, n_swap, seed, ties in cases:
        drho, ux, uy = _fields(cells.shape, seed, ties)
        lat = L.Lattice(cells, tau, 0.02)
        ref_f, ref_s = lat.select_swaps(drho, ux, uy, n_swap)
        lat.close()
        ora_f, ora_s = _oracle_pick(ora, cells, tau, drho, ux, uy, n_swap)
        st, n, got_f, got_s = _noalloc(lib, torch, cells, tau, drho, ux, uy, n_swap)
        assert st == 0, lib.lbm_last_error().decode()
        assert n == len(ref_f) == len(ref_s) == len(ora_f) == n_swap
        assert np.array_equal(got_f, ref_f) and np.array_equal(got_s, ref_s)
        assert np.array_equal(got_f, ora_f) and np.array_equal(got_s, ora_s)


def test_noalloc_edge_cases(ora):
    torch = _torch()
    lib = L.load_library()
    cells = I.config_t_junction()["cells"]
    tau = 0.8
    drho, ux, uy = _fields(cells.shape, 3, False)
    # more picks asked for than there are candidates: n = min(n_swap, |F|, |S|)
    big = cells.size
    ora_f, ora_s = _oracle_pick(ora, cells, tau, drho, ux, uy, big)
    lat = L.Lattice(cells, tau, 0.02)
    ref_f, ref_s = lat.select_swaps(drho, ux, uy, big)
    st, n, got_f, got_s = _noalloc(lib, torch, cells, tau, drho, ux, uy, big)
    assert st == 0, lib.lbm_last_error().decode()
    assert 0 < n == len(ora_f) == len(ref_f) < big
    assert np.array_equal(got_f, ora_f) and np.array_equal(got_s, ora_s)
    assert np.array_equal(got_f, ref_f) and np.array_equal(got_s, ref_s)
    # a NaN in the velocity of one fluid candidate: no picks, n_out = -1
    ny, nx = cells.shape
    p = ora.make_params(nx, ny, tau, 1.0)
    cand, _ = ora.scores(p, cells, 1.0 + drho.astype(np.float64), ux.astype(np.float64), uy.astype(np.float64))
    y, x = np.argwhere(cand == 1)[0]
    ux_nan = ux.copy()
    ux_nan[y, x] = np.nan
    st, n, _, _ = _noalloc(lib, torch, cells, tau, drho, ux_nan, uy, 5)
    assert st == 0 and n == -1
    with pytest.raises(L.LbmError):
        lat.select_swaps(drho, ux_nan, uy, 5)
    lat.close()
    # nothing asked for: no output buffers needed, n_out = 0
    st, n, _, _ = _noalloc(lib, torch, cells, tau, drho, ux, uy, 0, with_outputs=False)
    assert st == 0 and n == 0


def test_noalloc_rejects_lattices_beyond_its_scratch():
    torch = _torch()
    lib = L.load_library()
    one = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = one.data_ptr()
    # 1024 x 512 = 524288 cells > 262144: refused before any device work
    st = lib.lbm_select_swaps_noalloc(1024, 512, 0.8, 1.0, p, p, p, p, 4, p, p, p, None)
    assert st == 1 and b"scratch" in lib.lbm_last_error()
    st = lib.lbm_select_swaps_noalloc(8192, 8, 0.8, 1.0, p, p, p, p, 4, p, p, p, None)
    assert st == 1
