"""ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

Every computation runs in the CUDA library; this module converts numpy arrays
and torch tensors to pointers, structs to dicts, and status codes to
exceptions.  Importing it does not need a GPU; loading the library fails
loudly if it has not been built.
"""
import ctypes
import pathlib

import numpy as np

import os

from .build import LIB, LIB_CHECKED

F32, BF16_SHIFTED, F16_SHIFTED = 0, 1, 2
OUT_CONST_RHO, OUT_NEUMANN = 0, 1
PORTS_REGULARIZED, PORTS_ZOU_HE = 0, 1
REINIT_WARM, REINIT_COLD = 0, 1
FIELD_RHO, FIELD_UX, FIELD_UY, FIELD_MASK, FIELD_POPS, FIELD_DRHO = 1, 2, 4, 8, 16, 32
MAX_OUTLETS = 64
PRECISIONS = {"f32": F32, "bf16": BF16_SHIFTED, "f16": F16_SHIFTED}
STATUS = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_GEOMETRY", 3: "LBM_ERR_OOM", 4: "LBM_ERR_CUDA",
          5: "LBM_ERR_DIVERGED", 6: "LBM_ERR_TIMEOUT", 7: "LBM_ERR_BUSY"}


class LbmError(RuntimeError):
    def __init__(self, status, where, detail):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("tau", ctypes.c_double),
                ("rho0", ctypes.c_double), ("u_max", ctypes.c_double), ("outlet", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("reinit", ctypes.c_int32),
                ("residual_every", ctypes.c_int32), ("ports", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class SolveResult(ctypes.Structure):
    _fields_ = [("dp", ctypes.c_double), ("m_in", ctypes.c_double), ("residual", ctypes.c_double),
                ("n_outlets", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("m_out", ctypes.c_double * MAX_OUTLETS), ("theta", ctypes.c_double),
                ("dg", ctypes.c_double), ("steps_done", ctypes.c_int64), ("fluid_cells", ctypes.c_int64)]

    def to_dict(self):
        n = self.n_outlets
        return dict(dp=self.dp, m_in=self.m_in, residual=self.residual, n_outlets=n,
                    m_out=np.array(self.m_out[:n]), theta=self.theta, dg=self.dg,
                    steps_done=self.steps_done, fluid_cells=self.fluid_cells)


class OptResult(ctypes.Structure):
    _fields_ = [("n_swapped", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("fluid_count", ctypes.c_int64), ("solve", SolveResult)]


_LIB = None
_VP = ctypes.c_void_p


def load_library(path=None):
    """Load the built library (raises if it is missing: there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if path is None and os.environ.get("LBM_CHECKED") == "1":
        path = LIB_CHECKED
    p = pathlib.Path(path) if path else LIB
    if not p.exists():
        raise RuntimeError(f"CUDA library not built: {p} is missing; run paper_1303_0107_gb300.build.build()")
    L = ctypes.CDLL(str(p))
    H = _VP
    L.lbm_create_geometry.argtypes = [ctypes.POINTER(Params), _VP, _VP, ctypes.POINTER(H)]
    L.lbm_solve.argtypes = [H, ctypes.c_int64, ctypes.POINTER(SolveResult)]
    L.lbm_optimize_step.argtypes = [H, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(OptResult)]
    L.lbm_read_fields.argtypes = [H, ctypes.c_uint32, _VP, ctypes.c_size_t, ctypes.c_int]
    L.lbm_load_state.argtypes = [H, _VP, ctypes.c_size_t, ctypes.c_int]
    L.lbm_reset.argtypes = [H]
    L.lbm_select_swaps.argtypes = [H, _VP, _VP, _VP, ctypes.c_int32, _VP, _VP, ctypes.POINTER(ctypes.c_int32)]
    L.lbm_destroy.argtypes = [H]
    L.lbm_destroy.restype = None
    L.lbm_status_str.argtypes = [ctypes.c_int]
    L.lbm_status_str.restype = ctypes.c_char_p
    L.lbm_last_error.argtypes = []
    L.lbm_last_error.restype = ctypes.c_char_p
    L.lbm_kernel_launches.argtypes = []
    L.lbm_kernel_launches.restype = ctypes.c_uint64
    L.lbm_kernel_time.argtypes = [H, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.lbm_step_config.argtypes = [H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    B = _VP
    L.lbm_batch_create.argtypes = [ctypes.c_int32, ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_void_p), _VP,
                                   ctypes.POINTER(B)]
    L.lbm_batch_solve.argtypes = [B, ctypes.c_int64, ctypes.POINTER(SolveResult)]
    L.lbm_batch_optimize_step.argtypes = [B, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64,
                                          ctypes.POINTER(OptResult)]
    L.lbm_batch_read_fields.argtypes = [B, ctypes.c_int32, ctypes.c_uint32, _VP, ctypes.c_size_t, ctypes.c_int]
    L.lbm_batch_reset.argtypes = [B]
    L.lbm_batch_kernel_time.argtypes = [B, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.lbm_batch_step_config.argtypes = [B, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    L.lbm_batch_destroy.argtypes = [B]
    L.lbm_batch_destroy.restype = None
    L.lbm_select_swaps_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                           _VP, _VP, _VP, _VP, ctypes.c_int32, _VP, _VP, _VP, _VP]
    L.lbm_bytes_per_fluid_update.argtypes = [ctypes.c_int32]
    L.lbm_bytes_per_fluid_update.restype = ctypes.c_double
    for name in ("lbm_create_geometry", "lbm_solve", "lbm_optimize_step", "lbm_read_fields",
                 "lbm_load_state", "lbm_reset", "lbm_select_swaps", "lbm_kernel_time",
                 "lbm_select_swaps_noalloc", "lbm_step_config", "lbm_batch_create", "lbm_batch_solve",
                 "lbm_batch_optimize_step", "lbm_batch_read_fields", "lbm_batch_reset",
                 "lbm_batch_kernel_time", "lbm_batch_step_config"):
        getattr(L, name).restype = ctypes.c_int
    _LIB = L
    return L


def _check(st, where):
    if st != 0:
        raise LbmError(st, where, load_library().lbm_last_error().decode())


def kernel_launches() -> int:
    return int(load_library().lbm_kernel_launches())


def bytes_per_fluid_update(precision: int) -> float:
    return float(load_library().lbm_bytes_per_fluid_update(int(precision)))


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return int(stream.cuda_stream) or None  # torch.cuda.Stream


def _buffer(dst):
    """(pointer, nbytes, is_device) of a numpy array or torch tensor."""
    if isinstance(dst, np.ndarray):
        assert dst.flags.c_contiguous
        return dst.ctypes.data, dst.nbytes, 0
    import torch
    assert isinstance(dst, torch.Tensor) and dst.is_contiguous()
    return dst.data_ptr(), dst.numel() * dst.element_size(), int(dst.is_cuda)


class Lattice:
    """One lattice (cell map + populations) resident on the GPU."""

    def __init__(self, cells, tau, u_max, rho0=1.0, outlet=OUT_CONST_RHO, precision=F32,
                 reinit=REINIT_WARM, residual_every=100, stream=None, ports=PORTS_REGULARIZED):
        L = load_library()
        cells = np.ascontiguousarray(cells, dtype=np.uint8)
        ny, nx = cells.shape
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self.params = Params(nx, ny, float(tau), float(rho0), float(u_max), int(outlet), int(precision),
                             int(reinit), int(residual_every), int(ports), 0)
        self.nx, self.ny, self.precision = nx, ny, int(precision)
        self._h = _VP()
        _check(L.lbm_create_geometry(ctypes.byref(self.params), cells.ctypes.data, _stream_ptr(stream),
                                     ctypes.byref(self._h)), "lbm_create_geometry")

    def close(self):
        if self._h:
            load_library().lbm_destroy(self._h)
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
        r = SolveResult()
        _check(load_library().lbm_solve(self._h, int(n_steps), ctypes.byref(r)), "lbm_solve")
        return r.to_dict()

    def optimize_step(self, n_swap: int, n_steps: int) -> dict:
        r = OptResult()
        _check(load_library().lbm_optimize_step(self._h, int(n_swap), int(n_steps), ctypes.byref(r)),
               "lbm_optimize_step")
        out = r.solve.to_dict()
        out.update(n_swapped=r.n_swapped, fluid_count=r.fluid_count)
        return out

    def _field_shape_dtype(self, field):
        if field == FIELD_MASK:
            return (self.ny, self.nx), np.uint8
        if field == FIELD_POPS:
            return (9, self.ny, self.nx), (np.float32 if self.precision == F32 else np.uint16)
        return (self.ny, self.nx), np.float32

    def read(self, field: int, out=None):
        """Copy a field into `out` (numpy array or torch tensor; new numpy array if None)."""
        if out is None:
            shape, dt = self._field_shape_dtype(field)
            out = np.empty(shape, dt)
        ptr, nbytes, dev = _buffer(out)
        _check(load_library().lbm_read_fields(self._h, int(field), ptr, nbytes, dev), "lbm_read_fields")
        return out

    def load_state(self, pops):
        ptr, nbytes, dev = _buffer(pops)
        _check(load_library().lbm_load_state(self._h, ptr, nbytes, dev), "lbm_load_state")

    def kernel_time(self, reset=False):
        """(ms, launches, fluid_updates) of the stream-collide kernels, from CUDA events."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        u = ctypes.c_int64()
        _check(load_library().lbm_kernel_time(self._h, int(bool(reset)), ctypes.byref(ms), ctypes.byref(n),
                                              ctypes.byref(u)), "lbm_kernel_time")
        return ms.value, n.value, u.value

    def reset(self):
        _check(load_library().lbm_reset(self._h), "lbm_reset")

    def step_config(self):
        """(warps per block, blocks) of the time-step launches (autotuned)."""
        w = ctypes.c_int32()
        g = ctypes.c_int32()
        _check(load_library().lbm_step_config(self._h, ctypes.byref(w), ctypes.byref(g)), "lbm_step_config")
        return w.value, g.value

    def select_swaps(self, drho, ux, uy, n_swap: int):
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (drho, ux, uy)]
        cap = max(int(n_swap), 1)
        fi = np.zeros(cap, np.int32)
        si = np.zeros(cap, np.int32)
        n = ctypes.c_int32()
        _check(load_library().lbm_select_swaps(self._h, *[a.ctypes.data for a in arrs], int(n_swap),
                                               fi.ctypes.data, si.ctypes.data, ctypes.byref(n)),
               "lbm_select_swaps")
        return fi[:n.value].copy(), si[:n.value].copy()


class Batch:
    """Many lattices stepped together (one launch per stage for all of them).

    members: list of dicts with keys cells, tau, u_max and optionally rho0,
    outlet, ports, reinit.  precision and residual_every are shared.
    """

    def __init__(self, members, precision=F32, residual_every=100, stream=None):
        L = load_library()
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self.n = len(members)
        self.precision = int(precision)
        self._cells = [np.ascontiguousarray(m["cells"], dtype=np.uint8) for m in members]
        self.shapes = [c.shape for c in self._cells]
        params = (Params * self.n)()
        for i, m in enumerate(members):
            ny, nx = self._cells[i].shape
            params[i] = Params(nx, ny, float(m["tau"]), float(m.get("rho0", 1.0)), float(m["u_max"]),
                               int(m.get("outlet", OUT_CONST_RHO)), int(precision),
                               int(m.get("reinit", REINIT_WARM)), int(residual_every),
                               int(m.get("ports", PORTS_REGULARIZED)), 0)
        ptrs = (ctypes.c_void_p * self.n)(*[c.ctypes.data for c in self._cells])
        self._b = _VP()
        _check(L.lbm_batch_create(self.n, params, ptrs, _stream_ptr(stream), ctypes.byref(self._b)),
               "lbm_batch_create")

    def close(self):
        if self._b:
            load_library().lbm_batch_destroy(self._b)
            self._b = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, n_steps):
        r = (SolveResult * self.n)()
        _check(load_library().lbm_batch_solve(self._b, int(n_steps), r), "lbm_batch_solve")
        return [x.to_dict() for x in r]

    def optimize_step(self, n_swap, n_steps):
        if np.isscalar(n_swap):
            n_swap = [int(n_swap)] * self.n
        ns = (ctypes.c_int32 * self.n)(*[int(v) for v in n_swap])
        r = (OptResult * self.n)()
        _check(load_library().lbm_batch_optimize_step(self._b, ns, int(n_steps), r), "lbm_batch_optimize_step")
        out = []
        for x in r:
            d = x.solve.to_dict()
            d.update(n_swapped=x.n_swapped, fluid_count=x.fluid_count)
            out.append(d)
        return out

    def read(self, member, field, out=None):
        if not 0 <= int(member) < self.n:
            raise LbmError(1, "lbm_batch_read_fields", f"member {member} out of range (batch of {self.n})")
        ny, nx = self.shapes[member]
        if out is None:
            if field == FIELD_MASK:
                out = np.empty((ny, nx), np.uint8)
            elif field == FIELD_POPS:
                out = np.empty((9, ny, nx), np.float32 if self.precision == F32 else np.uint16)
            else:
                out = np.empty((ny, nx), np.float32)
        ptr, nbytes, dev = _buffer(out)
        _check(load_library().lbm_batch_read_fields(self._b, int(member), int(field), ptr, nbytes, dev),
               "lbm_batch_read_fields")
        return out

    def reset(self):
        _check(load_library().lbm_batch_reset(self._b), "lbm_batch_reset")

    def kernel_time(self, reset=False):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        u = ctypes.c_int64()
        _check(load_library().lbm_batch_kernel_time(self._b, int(bool(reset)), ctypes.byref(ms), ctypes.byref(n),
                                                    ctypes.byref(u)), "lbm_batch_kernel_time")
        return ms.value, n.value, u.value

    def step_config(self):
        w = ctypes.c_int32()
        g = ctypes.c_int32()
        _check(load_library().lbm_batch_step_config(self._b, ctypes.byref(w), ctypes.byref(g)),
               "lbm_batch_step_config")
        return w.value, g.value
