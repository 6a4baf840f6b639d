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
COLLIDE_BGK, COLLIDE_REGULARIZED, COLLIDE_SMAGORINSKY = 0, 1, 2
OUT_CONST_RHO, OUT_NEUMANN = 0, 1
PORTS_REGULARIZED, PORTS_ZOU_HE = 0, 1
REINIT_WARM, REINIT_COLD = 0, 1
FIELD_RHO, FIELD_UX, FIELD_UY, FIELD_MASK, FIELD_POPS, FIELD_DRHO = 1, 2, 4, 8, 16, 32
MAX_OUTLETS = 64
PRECISIONS = {"f32": F32, "bf16": BF16_SHIFTED, "f16": F16_SHIFTED}
STATUS = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_GEOMETRY", 3: "LBM_ERR_OOM", 4: "LBM_ERR_CUDA",
          5: "LBM_ERR_DIVERGED", 6: "LBM_ERR_TIMEOUT", 7: "LBM_ERR_BUSY", 8: "LBM_ERR_CANCELLED"}


class LbmError(RuntimeError):
    def __init__(self, status, where, detail):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("tau", ctypes.c_double),
                ("rho0", ctypes.c_double), ("u_max", ctypes.c_double), ("outlet", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("reinit", ctypes.c_int32),
                ("residual_every", ctypes.c_int32), ("ports", ctypes.c_int32), ("guard", ctypes.c_int32),
                ("collision", ctypes.c_int32), ("mirror", ctypes.c_int32), ("c_smag", ctypes.c_double)]


def make_params(nx, ny, tau, u_max, rho0=1.0, outlet=0, precision=0, reinit=0, residual_every=0, ports=0,
                guard=False, collision=0, c_smag=0.0, mirror=False):
    return Params(int(nx), int(ny), float(tau), float(rho0), float(u_max), int(outlet), int(precision),
                  int(reinit), int(residual_every), int(ports), int(bool(guard)), int(collision),
                  int(bool(mirror)), float(c_smag))


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


class OptPlan(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int64), ("max_iter", ctypes.c_int32), ("n_swap", ctypes.c_int32),
                ("tol", ctypes.c_double), ("patience", ctypes.c_int32), ("adapt", ctypes.c_int32),
                ("keep_best", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class OptSummary(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("best_iter", ctypes.c_int32), ("stopped", ctypes.c_int32),
                ("n_swap_final", ctypes.c_int32), ("swapped", ctypes.c_int64), ("dp_first", ctypes.c_double),
                ("dp_best", ctypes.c_double), ("dp_last", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_active", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64), ("max_tick_steps", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("params", Params), ("cell_types", ctypes.c_void_p), ("n_steps", ctypes.c_int64),
                ("n_iter", ctypes.c_int32), ("n_swap", ctypes.c_int32), ("tag", ctypes.c_int64),
                ("out_mask", ctypes.c_void_p), ("out_drho", ctypes.c_void_p), ("out_ux", ctypes.c_void_p),
                ("out_uy", ctypes.c_void_p)]


class Served(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_int64), ("status", ctypes.c_int32), ("n_swapped", ctypes.c_int32),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("fluid_updates", ctypes.c_int64), ("footprint_bytes", ctypes.c_int64),
                ("dp_first", ctypes.c_double), ("last", SolveResult)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("ticks", ctypes.c_int64), ("exchanges", ctypes.c_int64),
                ("fluid_updates", ctypes.c_int64), ("resident_bytes", ctypes.c_int64),
                ("peak_resident_bytes", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("peak_device_bytes", ctypes.c_int64), ("active", ctypes.c_int32),
                ("peak_active", ctypes.c_int32), ("queued", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("busy_s", ctypes.c_double), ("step_ms", ctypes.c_double), ("budget_bytes", ctypes.c_int64)]


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
    L.lbm_optimize.argtypes = [H, ctypes.POINTER(OptPlan), _VP, ctypes.POINTER(OptSummary)]
    L.lbm_load_state.argtypes = [H, _VP, ctypes.c_size_t, ctypes.c_int]
    L.lbm_reset.argtypes = [H]
    L.lbm_select_swaps.argtypes = [H, _VP, _VP, _VP, ctypes.c_int32, _VP, _VP, ctypes.POINTER(ctypes.c_int32)]
    L.lbm_destroy.argtypes = [H]
    L.lbm_destroy.restype = None
    L.lbm_transfer_bytes.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
    L.lbm_transfer_bytes.restype = None
    L.lbm_status_str.argtypes = [ctypes.c_int]
    L.lbm_status_str.restype = ctypes.c_char_p
    L.lbm_last_error.argtypes = []
    L.lbm_last_error.restype = ctypes.c_char_p
    L.lbm_kernel_launches.argtypes = []
    L.lbm_kernel_launches.restype = ctypes.c_uint64
    L.lbm_kernel_time.argtypes = [H, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.lbm_step_config.argtypes = [H] + [ctypes.POINTER(ctypes.c_int32)] * 5
    L.lbm_set_step_config.argtypes = [H, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
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
    L.lbm_batch_step_config.argtypes = [B] + [ctypes.POINTER(ctypes.c_int32)] * 5
    L.lbm_batch_step_groups.argtypes = [B, ctypes.c_void_p]
    L.lbm_batch_set_step_config.argtypes = [B, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    L.lbm_batch_destroy.argtypes = [B]
    L.lbm_batch_destroy.restype = None
    L.lbm_select_swaps_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                           _VP, _VP, _VP, _VP, ctypes.c_int32, _VP, _VP, _VP, _VP]
    S = _VP
    L.lbm_server_create.argtypes = [ctypes.POINTER(ServerConfig), _VP, ctypes.POINTER(S)]
    L.lbm_server_submit.argtypes = [S, ctypes.POINTER(Request)]
    L.lbm_server_poll.argtypes = [S, ctypes.POINTER(Served), ctypes.c_int32, ctypes.c_int32]
    L.lbm_server_poll.restype = ctypes.c_int32
    L.lbm_server_wait_idle.argtypes = [S, ctypes.c_int32]
    L.lbm_server_get_stats.argtypes = [S, ctypes.POINTER(ServerStats)]
    L.lbm_server_now.argtypes = [S]
    L.lbm_server_now.restype = ctypes.c_double
    L.lbm_server_footprint.argtypes = [ctypes.POINTER(Params), ctypes.c_int32]
    L.lbm_server_footprint.restype = ctypes.c_int64
    L.lbm_server_cancel.argtypes = [S, ctypes.c_int64]
    L.lbm_debug_fail_alloc.argtypes = [ctypes.c_int64]
    L.lbm_debug_fail_alloc.restype = None
    L.lbm_debug_barrier_timeout.argtypes = [ctypes.c_int32]
    L.lbm_debug_barrier_timeout.restype = None
    L.lbm_debug_damage_canary.argtypes = [H]
    L.lbm_debug_task_counts.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p]
    L.lbm_server_destroy.argtypes = [S]
    L.lbm_server_destroy.restype = None
    L.lbm_bytes_per_fluid_update.argtypes = [ctypes.c_int32]
    L.lbm_bytes_per_fluid_update.restype = ctypes.c_double
    for name in ("lbm_create_geometry", "lbm_solve", "lbm_optimize_step", "lbm_optimize", "lbm_read_fields",
                 "lbm_load_state", "lbm_reset", "lbm_select_swaps", "lbm_kernel_time",
                 "lbm_select_swaps_noalloc", "lbm_step_config", "lbm_set_step_config", "lbm_batch_create", "lbm_batch_solve",
                 "lbm_batch_optimize_step", "lbm_batch_read_fields", "lbm_batch_reset",
                 "lbm_batch_kernel_time", "lbm_batch_step_config", "lbm_batch_set_step_config", "lbm_server_create", "lbm_server_submit",
                 "lbm_server_wait_idle", "lbm_server_get_stats", "lbm_server_cancel"):
        getattr(L, name).restype = ctypes.c_int
    _LIB = L
    return L


def _check(st, where):
    if st != 0:
        raise LbmError(st, where, load_library().lbm_last_error().decode())


def debug_fail_alloc(after: int) -> None:
    """Make the device allocation after `after` more successful ones fail (test hook; -1: off)."""
    load_library().lbm_debug_fail_alloc(int(after))


def debug_barrier_timeout(on: bool) -> None:
    """Make the persistent kernel's grid barriers wait for an arrival that never
    comes, so that their bounded waits give up (test hook)."""
    load_library().lbm_debug_barrier_timeout(int(bool(on)))


def kernel_launches() -> int:
    return int(load_library().lbm_kernel_launches())


def transfer_bytes():
    """(host-to-device, device-to-host) bytes the library has copied in this process."""
    h2d, d2h = ctypes.c_uint64(), ctypes.c_uint64()
    load_library().lbm_transfer_bytes(ctypes.byref(h2d), ctypes.byref(d2h))
    return int(h2d.value), int(d2h.value)


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
                 reinit=REINIT_WARM, residual_every=100, stream=None, ports=PORTS_REGULARIZED, guard=False,
                 collision=COLLIDE_BGK, c_smag=0.0, mirror=False):
        L = load_library()
        cells = np.ascontiguousarray(cells, dtype=np.uint8)
        ny, nx = cells.shape
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self.params = make_params(nx, ny, tau, u_max, rho0, outlet, precision, reinit, residual_every, ports,
                                  guard, collision, c_smag, mirror)
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

    def optimize(self, n_steps, max_iter, n_swap, tol=0.0, patience=3, adapt=False, keep_best=False):
        """The whole loop of Sec. 2.3 (lbm_optimize): first solve, then up to
        max_iter exchange iterations; returns the summary with the dp history."""
        plan = OptPlan(int(n_steps), int(max_iter), int(n_swap), float(tol), int(patience), int(bool(adapt)),
                       int(bool(keep_best)), 0)
        hist = np.zeros(int(max_iter) + 1, np.float64)
        out = OptSummary()
        _check(load_library().lbm_optimize(self._h, ctypes.byref(plan), hist.ctypes.data, ctypes.byref(out)),
               "lbm_optimize")
        d = {k: getattr(out, k) for k, _ in OptSummary._fields_}
        d["history"] = hist[:out.iterations + 1].copy()
        return d

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
        """(warps per block, blocks, persistent, cells per thread, stages) of the time-step launches
        (autotuned)."""
        v = [ctypes.c_int32() for _ in range(5)]
        _check(load_library().lbm_step_config(self._h, *[ctypes.byref(x) for x in v]), "lbm_step_config")
        return tuple(x.value for x in v)

    def set_step_config(self, warps_per_block, persistent=False, cells_per_thread=1, stages=0):
        """Fix the launch shape instead of tuning it (lbm_set_step_config): warps per block 4, 8, 12,
        16 or 32 with one cell per thread, 4, 8, 12 or 24 with two; persistent 8 or 16 (8 with two
        cells); stages 0 (register loads) or 2 / 3 (shared-memory staging, one cell per thread, 4-16
        warps); persistent=2: on-chip resident steps (the shape follows from the lattice; the
        other arguments are ignored); persistent=3: compacted fluid-cell tasks (one cell per
        thread, 4-32 warps); persistent=4: paired tasks (interior 64-cell windows two cells a lane,
        cells_per_thread=2, 4, 8, 12 or 24 warps, stages 0 or 2-4).  Every shape computes the same values; LbmError
        (status 1) for any other shape, or for modes 2 - 4 on lattices they do not serve."""
        _check(load_library().lbm_set_step_config(self._h, int(warps_per_block), int(persistent),
                                                  int(cells_per_thread), int(stages)), "lbm_set_step_config")

    def task_counts(self):
        """(row segments holding fluid, interior 64-cell windows among them) of the work-list
        (lbm_debug_task_counts)."""
        seg = ctypes.c_int32()
        win = ctypes.c_int32()
        _check(load_library().lbm_debug_task_counts(self._h, ctypes.byref(seg), ctypes.byref(win)),
               "lbm_debug_task_counts")
        return seg.value, win.value

    def debug_damage_canary(self):
        """Bounds-checked build: overwrite part of a canary next to the populations (test hook)."""
        _check(load_library().lbm_debug_damage_canary(self._h), "lbm_debug_damage_canary")

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
            params[i] = make_params(nx, ny, m["tau"], m["u_max"], m.get("rho0", 1.0), m.get("outlet", OUT_CONST_RHO),
                                    precision, m.get("reinit", REINIT_WARM), residual_every,
                                    m.get("ports", PORTS_REGULARIZED), m.get("guard", False),
                                    m.get("collision", COLLIDE_BGK), m.get("c_smag", 0.0), m.get("mirror", False))
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
        """(warps per block, blocks, persistent, cells per thread, stages) of the batch's launches."""
        v = [ctypes.c_int32() for _ in range(5)]
        _check(load_library().lbm_batch_step_config(self._b, *[ctypes.byref(x) for x in v]), "lbm_batch_step_config")
        return tuple(x.value for x in v)

    def step_groups(self) -> int:
        """Member groups the time steps run in (lbm_batch_step_groups; 1: not grouped)."""
        n = ctypes.c_int32()
        _check(load_library().lbm_batch_step_groups(self._b, ctypes.byref(n)), "lbm_batch_step_groups")
        return n.value

    def set_step_config(self, warps_per_block, persistent=False, cells_per_thread=1, stages=0):
        """As Lattice.set_step_config, for every lattice of the batch."""
        _check(load_library().lbm_batch_set_step_config(self._b, int(warps_per_block), int(persistent),
                                                        int(cells_per_thread), int(stages)),
               "lbm_batch_set_step_config")


class Server:
    """Request loop with continuous batching (lbm_server_*).

    submit() queues a solve (n_iter = 0) or an optimisation (n_iter
    iterations after the first solve) of a geometry and returns at once; the
    library's scheduler thread admits requests by device footprint, steps all
    resident requests in the same launches, and poll() returns finished ones
    as dicts.  With keep_fields=True the final mask, drho, ux and uy come back
    in the result.
    """

    def __init__(self, precision=F32, max_active=256, hbm_budget_bytes=0, max_tick_steps=1000, stream=None):
        L = load_library()
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self.precision = int(precision)
        cfg = ServerConfig(int(precision), int(max_active), int(hbm_budget_bytes), int(max_tick_steps), 0)
        self._s = _VP()
        self._outs = {}
        _check(L.lbm_server_create(ctypes.byref(cfg), _stream_ptr(stream), ctypes.byref(self._s)),
               "lbm_server_create")

    @staticmethod
    def params_for(cells, tau, u_max, precision=F32, rho0=1.0, outlet=OUT_CONST_RHO, reinit=REINIT_WARM,
                   ports=PORTS_REGULARIZED, guard=False, collision=COLLIDE_BGK, c_smag=0.0, mirror=False):
        ny, nx = np.asarray(cells).shape
        return make_params(nx, ny, tau, u_max, rho0, outlet, precision, reinit, 0, ports, guard, collision, c_smag,
                           mirror)

    @staticmethod
    def footprint(nx, ny, n_iter=0, precision=F32):
        p = make_params(nx, ny, 0.6, 0.0, precision=precision)
        return int(load_library().lbm_server_footprint(ctypes.byref(p), int(n_iter)))

    def submit(self, tag, cells, tau, u_max, n_steps, n_iter=0, n_swap=0, keep_fields=False, **kw):
        cells = np.ascontiguousarray(cells, dtype=np.uint8)
        ny, nx = cells.shape
        r = Request()
        r.params = self.params_for(cells, tau, u_max, precision=self.precision, **kw)
        r.cell_types = cells.ctypes.data
        r.n_steps, r.n_iter, r.n_swap, r.tag = int(n_steps), int(n_iter), int(n_swap), int(tag)
        if keep_fields:
            outs = dict(mask=np.empty((ny, nx), np.uint8), drho=np.empty((ny, nx), np.float32),
                        ux=np.empty((ny, nx), np.float32), uy=np.empty((ny, nx), np.float32))
            r.out_mask, r.out_drho, r.out_ux, r.out_uy = [outs[k].ctypes.data for k in ("mask", "drho", "ux", "uy")]
            self._outs[int(tag)] = outs
        st = load_library().lbm_server_submit(self._s, ctypes.byref(r))
        if st != 0:
            self._outs.pop(int(tag), None)
        _check(st, "lbm_server_submit")

    def poll(self, max_out=256, wait_ms=0):
        buf = (Served * int(max_out))()
        k = load_library().lbm_server_poll(self._s, buf, int(max_out), int(wait_ms))
        out = []
        for x in buf[:k]:
            d = dict(tag=x.tag, status=x.status, n_swapped=x.n_swapped, t_submit=x.t_submit, t_admit=x.t_admit,
                     t_done=x.t_done, fluid_updates=x.fluid_updates, footprint_bytes=x.footprint_bytes,
                     dp_first=x.dp_first, last=x.last.to_dict())
            f = self._outs.pop(int(x.tag), None)
            if f is not None:
                d["fields"] = f
            out.append(d)
        return out

    def cancel(self, tag):
        _check(load_library().lbm_server_cancel(self._s, int(tag)), "lbm_server_cancel")

    def wait_idle(self, timeout_s=600.0):
        _check(load_library().lbm_server_wait_idle(self._s, int(timeout_s * 1000)), "lbm_server_wait_idle")

    def stats(self):
        st = ServerStats()
        _check(load_library().lbm_server_get_stats(self._s, ctypes.byref(st)), "lbm_server_get_stats")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_ if k != "reserved"}

    def now(self):
        return float(load_library().lbm_server_now(self._s))

    def close(self):
        if self._s:
            load_library().lbm_server_destroy(self._s)
            self._s = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
