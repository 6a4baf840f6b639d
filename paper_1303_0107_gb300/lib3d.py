"""ctypes binding of the D3Q19 C ABI in include/lbm3d.h (argument marshalling
only; every computation runs in the CUDA library)."""
import ctypes

import numpy as np

from .lib import (F32, MAX_OUTLETS, PRECISIONS, REINIT_WARM, OptPlan, OptSummary, _VP, _buffer, _check,
                  _stream_ptr, load_library)

FIELD3_DRHO, FIELD3_UX, FIELD3_UY, FIELD3_UZ, FIELD3_MASK, FIELD3_POPS = 1, 2, 4, 8, 16, 32
Q3 = 19


class Params3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
                ("u_max", ctypes.c_double), ("reinit", ctypes.c_int32), ("collision", ctypes.c_int32),
                ("c_smag", ctypes.c_double), ("mirror", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class SolveResult3(ctypes.Structure):
    _fields_ = [("dp", ctypes.c_double), ("m_in", ctypes.c_double), ("n_outlets", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("m_out", ctypes.c_double * MAX_OUTLETS),
                ("steps_done", ctypes.c_int64), ("fluid_cells", ctypes.c_int64)]

    def to_dict(self):
        n = self.n_outlets
        return dict(dp=self.dp, m_in=self.m_in, n_outlets=n, m_out=np.array(self.m_out[:n]),
                    steps_done=self.steps_done, fluid_cells=self.fluid_cells)


class OptResult3(ctypes.Structure):
    _fields_ = [("n_swapped", ctypes.c_int32), ("reserved", ctypes.c_int32), ("fluid_count", ctypes.c_int64),
                ("solve", SolveResult3)]


_bound = False


def _lib():
    global _bound
    L = load_library()
    if not _bound:
        H = _VP
        I32P = ctypes.POINTER(ctypes.c_int32)
        L.lbm3d_create.argtypes = [ctypes.POINTER(Params3), _VP, _VP, ctypes.POINTER(H)]
        L.lbm3d_destroy.argtypes = [H]
        L.lbm3d_destroy.restype = None
        L.lbm3d_solve.argtypes = [H, ctypes.c_int64, ctypes.POINTER(SolveResult3)]
        L.lbm3d_optimize_step.argtypes = [H, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(OptResult3)]
        L.lbm3d_read_fields.argtypes = [H, ctypes.c_uint32, _VP, ctypes.c_size_t, ctypes.c_int]
        L.lbm3d_load_state.argtypes = [H, _VP, ctypes.c_size_t, ctypes.c_int]
        L.lbm3d_select_swaps.argtypes = [H, _VP, _VP, _VP, _VP, ctypes.c_int32, _VP, _VP, I32P]
        L.lbm3d_kernel_time.argtypes = [H, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.lbm3d_set_block.argtypes = [H, ctypes.c_int32]
        L.lbm3d_debug_task_counts.argtypes = [H, I32P, I32P]
        L.lbm3d_optimize.argtypes = [H, ctypes.POINTER(OptPlan), _VP, ctypes.POINTER(OptSummary)]
        for name in ("lbm3d_create", "lbm3d_solve", "lbm3d_optimize_step", "lbm3d_read_fields", "lbm3d_load_state",
                     "lbm3d_select_swaps", "lbm3d_kernel_time", "lbm3d_set_block", "lbm3d_optimize",
                     "lbm3d_debug_task_counts"):
            getattr(L, name).restype = ctypes.c_int
        _bound = True
    return L


def make_params3(nx, ny, nz, tau, u_max, rho0=1.0, precision=F32, reinit=REINIT_WARM, collision=0, c_smag=0.0,
                 mirror=False):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    return Params3(int(nx), int(ny), int(nz), int(precision), float(tau), float(rho0), float(u_max), int(reinit),
                   int(collision), float(c_smag), int(mirror), 0)


class Lattice3:
    """One D3Q19 lattice (cell map [nz][ny][nx] + populations) resident on the GPU.

    mirror: bit 0 a symmetry plane below y = 0, bit 1 one below z = 0 (True = bit 0)."""

    def __init__(self, cells, tau, u_max, rho0=1.0, precision=F32, reinit=REINIT_WARM, collision=0, c_smag=0.0,
                 mirror=False, stream=None):
        L = _lib()
        cells = np.ascontiguousarray(cells, dtype=np.uint8)
        self.nz, self.ny, self.nx = cells.shape
        self.params = make_params3(self.nx, self.ny, self.nz, tau, u_max, rho0, precision, reinit, collision, c_smag,
                                   mirror)
        self.precision = int(self.params.precision)
        self._h = _VP()
        _check(L.lbm3d_create(ctypes.byref(self.params), cells.ctypes.data, _stream_ptr(stream),
                              ctypes.byref(self._h)), "lbm3d_create")

    def close(self):
        if self._h:
            _lib().lbm3d_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, n_steps: int) -> dict:
        r = SolveResult3()
        _check(_lib().lbm3d_solve(self._h, int(n_steps), ctypes.byref(r)), "lbm3d_solve")
        return r.to_dict()

    def optimize_step(self, n_swap: int, n_steps: int) -> dict:
        r = OptResult3()
        _check(_lib().lbm3d_optimize_step(self._h, int(n_swap), int(n_steps), ctypes.byref(r)),
               "lbm3d_optimize_step")
        out = r.solve.to_dict()
        out.update(n_swapped=r.n_swapped, fluid_count=r.fluid_count)
        return out

    def optimize(self, n_steps, max_iter, n_swap, tol=0.0, patience=3, adapt=False, keep_best=False):
        """The whole loop of Sec. 2.3 (lbm3d_optimize); returns the summary with the dp history."""
        plan = OptPlan(int(n_steps), int(max_iter), int(n_swap), float(tol), int(patience), int(bool(adapt)),
                       int(bool(keep_best)), 0)
        hist = np.zeros(int(max_iter) + 1, np.float64)
        out = OptSummary()
        _check(_lib().lbm3d_optimize(self._h, ctypes.byref(plan), hist.ctypes.data, ctypes.byref(out)),
               "lbm3d_optimize")
        d = {k: getattr(out, k) for k, _ in OptSummary._fields_}
        d["history"] = hist[:out.iterations + 1].copy()
        return d

    def _shape_dtype(self, field):
        cells = (self.nz, self.ny, self.nx)
        if field == FIELD3_MASK:
            return cells, np.uint8
        if field == FIELD3_POPS:
            return (Q3,) + cells, (np.float32 if self.precision == F32 else np.uint16)
        return cells, np.float32

    def read(self, field: int, out=None):
        if out is None:
            shape, dt = self._shape_dtype(field)
            out = np.empty(shape, dt)
        ptr, nbytes, dev = _buffer(out)
        _check(_lib().lbm3d_read_fields(self._h, int(field), ptr, nbytes, dev), "lbm3d_read_fields")
        return out

    def load_state(self, pops):
        ptr, nbytes, dev = _buffer(pops)
        _check(_lib().lbm3d_load_state(self._h, ptr, nbytes, dev), "lbm3d_load_state")

    def select_swaps(self, drho, ux, uy, uz, n_swap: int):
        arrs = [np.ascontiguousarray(a, np.float32) for a in (drho, ux, uy, uz)]
        cap = max(int(n_swap), 1)
        fi = np.zeros(cap, np.int32)
        si = np.zeros(cap, np.int32)
        n = ctypes.c_int32()
        _check(_lib().lbm3d_select_swaps(self._h, *[a.ctypes.data for a in arrs], int(n_swap), fi.ctypes.data,
                                         si.ctypes.data, ctypes.byref(n)), "lbm3d_select_swaps")
        return fi[:n.value].copy(), si[:n.value].copy()

    def kernel_time(self, reset=False):
        """(ms, launches, fluid_updates) of the stream-collide kernels, from CUDA events."""
        ms, n, u = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib().lbm3d_kernel_time(self._h, int(bool(reset)), ctypes.byref(ms), ctypes.byref(n),
                                        ctypes.byref(u)), "lbm3d_kernel_time")
        return ms.value, n.value, u.value

    def set_block(self, warps_per_block: int):
        _check(_lib().lbm3d_set_block(self._h, int(warps_per_block)), "lbm3d_set_block")

    def task_counts(self):
        """(row-segment tasks, packed-cell tasks) of the current work-list."""
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib().lbm3d_debug_task_counts(self._h, ctypes.byref(a), ctypes.byref(b)), "lbm3d_debug_task_counts")
        return a.value, b.value
