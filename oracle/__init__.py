"""FP64 CPU oracle of the LBM shape-optimisation hot path (arXiv:1303.0107).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark load this package; the product path never does.  It shares
no code with the CUDA library: the arithmetic lives in lbm_oracle.c (plain C,
FP64, no contraction), and this module only marshals numpy arrays into it,
plus the plain host-side loop of Sec. 2.3 (solve, exchange, re-solve).
"""
import ctypes
import pathlib

import numpy as np

from . import build as _build
from .scaling import eq8_widths, reynolds, viscosity  # noqa: F401

OUT_CONST_RHO, OUT_NEUMANN = 0, 1
PORTS_REGULARIZED, PORTS_ZOU_HE = 0, 1
REINIT_WARM, REINIT_COLD = 0, 1
COLLIDE_BGK, COLLIDE_REGULARIZED, COLLIDE_SMAGORINSKY = 0, 1, 2


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("tau", ctypes.c_double),
                ("rho0", ctypes.c_double), ("u_max", ctypes.c_double),
                ("outlet_rule", ctypes.c_int32), ("periodic", ctypes.c_int32),
                ("port_scheme", ctypes.c_int32), ("guard", ctypes.c_int32), ("collision", ctypes.c_int32),
                ("mirror", ctypes.c_int32), ("c_smag", ctypes.c_double)]


_LIB = None
_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_I32 = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(str(path))
        P = ctypes.POINTER(Params)
        L.ora_lattice.argtypes = [_I32, _I32, _I32, _D, _D]
        L.ora_feq.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.ora_feq.restype = ctypes.c_double
        L.ora_inlet_profile.argtypes = [P, _U8, _D]
        L.ora_inlet_profile.restype = ctypes.c_int32
        L.ora_outlet_ids.argtypes = [P, _U8, _I32]
        L.ora_outlet_ids.restype = ctypes.c_int32
        L.ora_check_geometry.argtypes = [P, _U8]
        L.ora_check_geometry.restype = ctypes.c_int32
        L.ora_init.argtypes = [P, _U8, _D]
        L.ora_init_state.argtypes = [P, _U8, _D, _D, _D, _D]
        L.ora_step_columns.argtypes = [P, _U8, _D, _D, _D, _D, _D, _D, ctypes.c_int32, ctypes.c_int32]
        L.ora_step.argtypes = [P, _U8, _D, _D, _D, _D, _D, _D]
        L.ora_run.argtypes = [P, _U8, _D, _D, _D, ctypes.c_int64, _D, _D, _D]
        L.ora_run.restype = ctypes.c_int32
        L.ora_observables.argtypes = [P, _U8, _D, _D, _I32, ctypes.c_int32, _D, _D, _D]
        L.ora_observables.restype = ctypes.c_int32
        L.ora_uniformity.argtypes = [_D, ctypes.c_int32, _D, _D]
        L.ora_residual.argtypes = [P, _U8, _D, _D, _D, _D]
        L.ora_residual.restype = ctypes.c_double
        L.ora_scores.argtypes = [P, _U8, _D, _D, _D, ctypes.c_double, _U8, _D]
        L.ora_simple.argtypes = [P, _U8, ctypes.c_int32, ctypes.c_int32]
        L.ora_set_threads.argtypes = [ctypes.c_int32]
        L.ora_set_threads.restype = ctypes.c_int32
        L.ora_smagorinsky_tau.argtypes = [ctypes.c_double] * 6
        L.ora_smagorinsky_tau.restype = ctypes.c_double
        L.ora_simple.restype = ctypes.c_int32
        L.ora_select.argtypes = [P, _U8, _D, ctypes.c_int32, _I32, _I32, _I32]
        L.ora_select.restype = ctypes.c_int32
        L.ora_apply.argtypes = [P, _U8, _D, _I32, _I32, ctypes.c_int32, ctypes.c_int32]
        L.ora_apply.restype = ctypes.c_int64
        _LIB = L
    return _LIB


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def make_params(nx, ny, tau, rho0=1.0, u_max=0.0, outlet_rule=OUT_CONST_RHO, periodic=False,
                port_scheme=PORTS_REGULARIZED, guard=False, collision=0, c_smag=0.0, mirror=False):
    return Params(int(nx), int(ny), float(tau), float(rho0), float(u_max), int(outlet_rule),
                  int(bool(periodic)), int(port_scheme), int(bool(guard)), int(collision), int(bool(mirror)),
                  float(c_smag))


def lattice():
    """(cx, cy, opp, w, cs2) exactly as the oracle stores them."""
    cx = np.zeros(9, np.int32)
    cy = np.zeros(9, np.int32)
    opp = np.zeros(9, np.int32)
    w = np.zeros(9, np.float64)
    cs2 = ctypes.c_double()
    lib().ora_lattice(_p(cx, ctypes.c_int32), _p(cy, ctypes.c_int32), _p(opp, ctypes.c_int32),
                      _p(w, ctypes.c_double), ctypes.byref(cs2))
    return cx, cy, opp, w, cs2.value


def feq(i, rho, ux, uy):
    return lib().ora_feq(int(i), float(rho), float(ux), float(uy))


def inlet_profile(params, solid):
    u = np.zeros(params.ny, np.float64)
    lib().ora_inlet_profile(ctypes.byref(params), _p(_u8(solid), ctypes.c_uint8), _p(u, ctypes.c_double))
    return u


def outlet_ids(params, solid):
    ids = np.zeros(params.ny, np.int32)
    n = lib().ora_outlet_ids(ctypes.byref(params), _p(_u8(solid), ctypes.c_uint8), _p(ids, ctypes.c_int32))
    return ids, n


def check_geometry(params, solid):
    return lib().ora_check_geometry(ctypes.byref(params), _p(_u8(solid), ctypes.c_uint8))


def init(params, solid):
    f = np.zeros((9, params.ny, params.nx), np.float64)
    lib().ora_init(ctypes.byref(params), _p(_u8(solid), ctypes.c_uint8), _p(f, ctypes.c_double))
    return f


def init_state(params, solid, rho, ux, uy):
    f = np.zeros((9, params.ny, params.nx), np.float64)
    rho, ux, uy = _f64(rho), _f64(ux), _f64(uy)
    lib().ora_init_state(ctypes.byref(params), _p(_u8(solid), ctypes.c_uint8), _p(rho, ctypes.c_double),
                         _p(ux, ctypes.c_double), _p(uy, ctypes.c_double), _p(f, ctypes.c_double))
    return f


def step_columns(params, solid, u_in, f_post, x_begin, x_end, f_next=None, fields=None):
    """One time step over columns [x_begin, x_end) into f_next (returned)."""
    solid = _u8(solid)
    f_post = _f64(f_post)
    if f_next is None:
        f_next = np.zeros_like(f_post)
    if fields is None:
        fields = [np.zeros((params.ny, params.nx)) for _ in range(3)]
    lib().ora_step_columns(ctypes.byref(params), _p(solid, ctypes.c_uint8), _p(_f64(u_in), ctypes.c_double),
                           _p(f_post, ctypes.c_double), _p(f_next, ctypes.c_double),
                           *[_p(a, ctypes.c_double) for a in fields], int(x_begin), int(x_end))
    return f_next, fields


def run(params, solid, u_in, f, n_steps):
    """Advance the post-collision state f (copied) by n_steps; returns (f, rho, ux, uy, status)."""
    solid = _u8(solid)
    f = _f64(f).copy()
    work = np.zeros_like(f)
    rho = np.zeros((params.ny, params.nx))
    ux = np.zeros_like(rho)
    uy = np.zeros_like(rho)
    st = lib().ora_run(ctypes.byref(params), _p(solid, ctypes.c_uint8), _p(_f64(u_in), ctypes.c_double),
                       _p(f, ctypes.c_double), _p(work, ctypes.c_double), int(n_steps),
                       _p(rho, ctypes.c_double), _p(ux, ctypes.c_double), _p(uy, ctypes.c_double))
    return f, rho, ux, uy, st


def observables(params, solid, rho, ux):
    """(dp, m_in, m_out[]) of a solved field."""
    solid = _u8(solid)
    ids, n = outlet_ids(params, solid)
    m_out = np.zeros(max(n, 1))
    dp = ctypes.c_double()
    m_in = ctypes.c_double()
    st = lib().ora_observables(ctypes.byref(params), _p(solid, ctypes.c_uint8), _p(_f64(rho), ctypes.c_double),
                               _p(_f64(ux), ctypes.c_double), _p(ids, ctypes.c_int32), n,
                               ctypes.byref(dp), ctypes.byref(m_in), _p(m_out, ctypes.c_double))
    if st != 0:
        raise RuntimeError(f"observables failed with status {st}")
    return dp.value, m_in.value, m_out[:n].copy()


def uniformity(m):
    """(theta, D_g) of Eq. 9-10 for the outlet flow rates m."""
    m = _f64(m)
    th = ctypes.c_double()
    dg = ctypes.c_double()
    lib().ora_uniformity(_p(m, ctypes.c_double), len(m), ctypes.byref(th), ctypes.byref(dg))
    return th.value, dg.value


def residual(params, solid, ux, uy, ux_prev, uy_prev):
    return lib().ora_residual(ctypes.byref(params), _p(_u8(solid), ctypes.c_uint8),
                              *[_p(_f64(a), ctypes.c_double) for a in (ux, uy, ux_prev, uy_prev)])


def simple(params, solid, x, y):
    """1 if interior fluid cell (x, y) may turn solid under the connectivity guard."""
    return int(lib().ora_simple(ctypes.byref(params), _p(_u8(solid), ctypes.c_uint8), int(x), int(y)))


def set_threads(n):
    """Host threads of the time steps (n <= 0: leave as is); returns the number in force."""
    return int(lib().ora_set_threads(int(n)))


def mu_of(params):
    """Dynamic viscosity mu = rho0 nu with nu = (tau - 1/2)/3."""
    return params.rho0 * ((params.tau - 0.5) / 3.0)


def scores(params, solid, rho, ux, uy):
    """(cand, score): cand 1 = interface fluid, 2 = interface solid (Eq. 5, Eq. 6)."""
    cand = np.zeros((params.ny, params.nx), np.uint8)
    score = np.zeros((params.ny, params.nx))
    lib().ora_scores(ctypes.byref(params), _p(_u8(solid), ctypes.c_uint8),
                     *[_p(_f64(a), ctypes.c_double) for a in (rho, ux, uy)], mu_of(params),
                     _p(cand, ctypes.c_uint8), _p(score, ctypes.c_double))
    return cand, score


def select(params, cand, score, n_swap):
    """(fluid_idx, solid_idx) chosen for exchange, each sorted ascending."""
    cap = int(max(n_swap, 0))
    fi = np.zeros(max(cap, 1), np.int32)
    si = np.zeros(max(cap, 1), np.int32)
    n = ctypes.c_int32()
    st = lib().ora_select(ctypes.byref(params), _p(_u8(cand), ctypes.c_uint8), _p(_f64(score), ctypes.c_double),
                          int(n_swap), _p(fi, ctypes.c_int32), _p(si, ctypes.c_int32), ctypes.byref(n))
    if st != 0:
        raise RuntimeError(f"select failed with status {st}")
    return fi[:n.value].copy(), si[:n.value].copy()


def apply(params, solid, f, fluid_idx, solid_idx, reinit=REINIT_WARM):
    """Exchange in place (solid: uint8 array, f: float64 array); returns the fluid count."""
    assert solid.dtype == np.uint8 and solid.flags.c_contiguous
    assert f.dtype == np.float64 and f.flags.c_contiguous
    fi = np.ascontiguousarray(fluid_idx, np.int32)
    si = np.ascontiguousarray(solid_idx, np.int32)
    assert len(fi) == len(si)
    return lib().ora_apply(ctypes.byref(params), _p(solid, ctypes.c_uint8), _p(f, ctypes.c_double),
                           _p(fi, ctypes.c_int32), _p(si, ctypes.c_int32), len(fi), int(reinit))


def run_plan(solve, step, n_swap, max_iter, tol=0.0, patience=3, adapt=False):
    """The outer loop of Sec. 2.3 with its stopping test (step 5, "the pressure
    drop tends to extremum") read as: stop after an iteration once
    |dp_k - dp_(k-1)| <= tol |dp_k| has held on `patience` consecutive
    iterations (tol <= 0: run max_iter iterations).  With adapt, n_swap is
    halved (down to 1) after every iteration that raised dp.  The lowest dp
    (earliest on ties) is the best.

    solve() -> dp of the first solve; step(n_swap) -> dp after one exchange and
    re-solve.  Returns the history and the decisions."""
    hist = [solve()]
    best, calm, stopped = 0, 0, False
    for k in range(1, max_iter + 1):
        dp = step(n_swap)
        hist.append(dp)
        if dp < hist[best]:
            best = k
        if adapt and dp > hist[k - 1]:
            n_swap = max(1, n_swap // 2)
        if tol > 0:
            calm = calm + 1 if abs(dp - hist[k - 1]) <= tol * abs(dp) else 0
            if calm >= patience:
                stopped = True
                break
    return dict(history=hist, best_iter=best, dp_best=hist[best], stopped=stopped, n_swap_final=n_swap,
                iterations=len(hist) - 1)


class Solver:
    """The loop of Sec. 2.3 on the oracle: solve, pick and exchange, re-solve.

    State between calls is the post-collision lattice, as in the CUDA library.
    """

    def __init__(self, params, cell_types, reinit=REINIT_WARM, residual_every=100):
        self.params = params
        self.solid = _u8(cell_types).copy()
        st = check_geometry(params, self.solid)
        if st != 0:
            raise ValueError(f"geometry rejected ({st})")
        self.u_in = inlet_profile(params, self.solid)
        self.f = init(params, self.solid)
        self.reinit = reinit
        self.residual_every = residual_every
        self.rho = self.ux = self.uy = None
        self.steps_done = 0

    def solve(self, n_steps):
        K = self.residual_every
        res = float("nan")
        if K > 0 and n_steps >= K:
            f, _, uxp, uyp, st = run(self.params, self.solid, self.u_in, self.f, n_steps - K)
            f, rho, ux, uy, st2 = run(self.params, self.solid, self.u_in, f, K)
            st = st or st2
            if st == 0:
                res = residual(self.params, self.solid, ux, uy, uxp, uyp)
        else:
            f, rho, ux, uy, st = run(self.params, self.solid, self.u_in, self.f, n_steps)
        if st != 0:
            raise FloatingPointError("oracle diverged")
        self.f, self.rho, self.ux, self.uy = f, rho, ux, uy
        self.steps_done += n_steps
        dp, m_in, m_out = observables(self.params, self.solid, rho, ux)
        theta, dg = uniformity(m_out) if len(m_out) else (float("nan"), float("nan"))
        return dict(dp=dp, m_in=m_in, m_out=m_out, theta=theta, dg=dg, residual=res,
                    steps_done=self.steps_done)

    def pick(self, n_swap, rho=None, ux=None, uy=None):
        rho = self.rho if rho is None else rho
        ux = self.ux if ux is None else ux
        uy = self.uy if uy is None else uy
        cand, score = scores(self.params, self.solid, rho, ux, uy)
        return select(self.params, cand, score, n_swap)

    def exchange(self, fluid_idx, solid_idx):
        return apply(self.params, self.solid, self.f, fluid_idx, solid_idx, self.reinit)

    def optimize_step(self, n_swap, n_steps):
        fi, si = self.pick(n_swap)
        fluid = self.exchange(fi, si)
        out = self.solve(n_steps)
        out.update(n_swapped=len(fi), fluid_count=fluid, fluid_idx=fi, solid_idx=si)
        return out

    def _state(self):
        return (self.solid.copy(), self.f.copy(), self.rho.copy(), self.ux.copy(), self.uy.copy())

    def optimize_run(self, n_steps, max_iter, n_swap, tol=0.0, patience=3, adapt=False, keep_best=False):
        """run_plan on this solver; with keep_best the solver ends in the state
        of the best iteration."""
        saved = {}

        def solve():
            dp = self.solve(n_steps)["dp"]
            saved[0] = self._state()
            return dp

        def step(ns):
            dp = self.optimize_step(ns, n_steps)["dp"]
            saved[len(saved)] = self._state()
            return dp

        out = run_plan(solve, step, n_swap, max_iter, tol, patience, adapt)
        if keep_best:
            self.solid, self.f, self.rho, self.ux, self.uy = saved[out["best_iter"]]
        return out
