"""The exchange selection for callers that cannot allocate device memory.

Code that runs inside an application whose memory pool owns the GPU, or a
loop that must not risk the device-wide synchronisation of cudaMalloc and
cudaFree, cannot use the handle-based entry points (creating a handle
allocates).  lbm_select_swaps_noalloc takes only caller-owned device buffers
and keeps its intermediate data in a static device array.  Here it is called
through the C ABI twice in a row, on two lattices of different shapes (so
anything left over in the shared array from the first call would show), and
its picks must equal those of lbm_select_swaps bit for bit.  This file is
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


def test_noalloc_selection_equals_handle_selection_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = L.load_library()
    t_junction = I.config_t_junction()
    cases = [(t_junction["cells"], t_junction["tau"], 7, 0, False),
             (I.random_blobs(100, 40, 5, density=0.3), 0.7, 25, 1, True)]
    stream = torch.cuda.current_stream()
    for cells, tau, n_swap, seed, ties in cases:
        ny, nx = cells.shape
        drho, ux, uy = _fields(cells.shape, seed, ties)
        lat = L.Lattice(cells, tau, 0.02)
        ref_f, ref_s = lat.select_swaps(drho, ux, uy, n_swap)
        lat.close()
        dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (cells, drho, ux, uy)]
        out_f = torch.full((n_swap,), -7, dtype=torch.int32, device="cuda")
        out_s = torch.full((n_swap,), -7, dtype=torch.int32, device="cuda")
        n_dev = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        st = lib.lbm_select_swaps_noalloc(nx, ny, tau, 1.0, *[t.data_ptr() for t in dev], n_swap,
                                          out_f.data_ptr(), out_s.data_ptr(), n_dev.data_ptr(),
                                          stream.cuda_stream)
        assert st == 0, lib.lbm_last_error().decode()
        torch.cuda.synchronize()
        n = int(n_dev.item())
        assert n == len(ref_f) == len(ref_s)
        assert np.array_equal(out_f[:n].cpu().numpy(), ref_f)
        assert np.array_equal(out_s[:n].cpu().numpy(), ref_s)


def test_noalloc_rejects_lattices_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = L.load_library()
    one = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = one.data_ptr()
    # 1024 x 512 = 524288 cells > 262144: refused before any device work
    st = lib.lbm_select_swaps_noalloc(1024, 512, 0.8, 1.0, p, p, p, p, 4, p, p, p, None)
    assert st == 1 and b"scratch" in lib.lbm_last_error()
    st = lib.lbm_select_swaps_noalloc(8192, 8, 0.8, 1.0, p, p, p, p, 4, p, p, p, None)
    assert st == 1
