"""Python side of the D3Q19 oracle (lbm3d_oracle.c): ctypes marshalling and
the plain loop of Sec. 2.3 in 3D.  TEST INFRASTRUCTURE ONLY, like the 2D
oracle: only tests, the smoke check and the benchmark's CPU legs load it."""
import ctypes

import numpy as np

from . import lib, make_params, select, REINIT_WARM


COLLIDE_BGK, COLLIDE_REGULARIZED, COLLIDE_SMAGORINSKY = 0, 1, 2


class Params3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("periodic", ctypes.c_int32), ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
                ("u_max", ctypes.c_double), ("collision", ctypes.c_int32), ("mirror", ctypes.c_int32),
                ("c_smag", ctypes.c_double)]


_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_I32 = ctypes.POINTER(ctypes.c_int32)
_ready = False


def _lib():
    global _ready
    L = lib()
    if not _ready:
        P = ctypes.POINTER(Params3)
        L.ora3_lattice.argtypes = [_I32, _I32, _I32, _I32, _D, _D]
        L.ora3_feq.argtypes = [ctypes.c_int32] + [ctypes.c_double] * 4
        L.ora3_feq.restype = ctypes.c_double
        L.ora3_check_geometry.argtypes = [P, _U8]
        L.ora3_check_geometry.restype = ctypes.c_int32
        L.ora3_inlet_profile.argtypes = [P, _U8, _D]
        L.ora3_outlet_ids.argtypes = [P, _U8, _I32]
        L.ora3_outlet_ids.restype = ctypes.c_int32
        L.ora3_init.argtypes = [P, _U8, _D]
        L.ora3_init_state.argtypes = [P, _U8, _D, _D, _D, _D, _D]
        L.ora3_run.argtypes = [P, _U8, _D, _D, _D, ctypes.c_int64, _D, _D, _D, _D]
        L.ora3_run.restype = ctypes.c_int32
        L.ora3_observables.argtypes = [P, _U8, _D, _D, _I32, ctypes.c_int32, _D, _D, _D]
        L.ora3_scores.argtypes = [P, _U8, _D, _D, _D, _D, ctypes.c_double, _U8, _D]
        L.ora3_apply.argtypes = [P, _U8, _D, _I32, _I32, ctypes.c_int32, ctypes.c_int32]
        L.ora3_apply.restype = ctypes.c_int64
        L.ora3_regularize.argtypes = [_D] + [ctypes.c_double] * 4
        L.ora3_collide.argtypes = [P, _D]
        L.ora3_collide.restype = ctypes.c_double
        _ready = True
    return L


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def make_params3(nx, ny, nz, tau, rho0=1.0, u_max=0.0, periodic=0, collision=COLLIDE_BGK, c_smag=0.0,
                 mirror=0):
    """mirror: bit 0 a symmetry plane below y = 0, bit 1 one below z = 0 (True = bit 0)."""
    return Params3(int(nx), int(ny), int(nz), int(periodic), float(tau), float(rho0), float(u_max), int(collision),
                   int(mirror), float(c_smag))


def collide3(p, f):
    """One cell's moments and collision (a copy); returns (f_post, tau_eff)."""
    f = np.ascontiguousarray(f, np.float64).copy()
    tau = _lib().ora3_collide(ctypes.byref(p), _p(f, ctypes.c_double))
    return f, tau


def lattice3():
    cx, cy, cz, opp = (np.zeros(19, np.int32) for _ in range(4))
    w = np.zeros(19)
    cs2 = ctypes.c_double()
    _lib().ora3_lattice(_p(cx, ctypes.c_int32), _p(cy, ctypes.c_int32), _p(cz, ctypes.c_int32),
                        _p(opp, ctypes.c_int32), _p(w, ctypes.c_double), ctypes.byref(cs2))
    return cx, cy, cz, opp, w, cs2.value


def feq3(i, rho, ux, uy, uz):
    return _lib().ora3_feq(int(i), float(rho), float(ux), float(uy), float(uz))


def regularize3(f, rho, ux, uy, uz):
    """The port cells' regularisation of the 19 populations f (a copy)."""
    f = np.ascontiguousarray(f, np.float64).copy()
    _lib().ora3_regularize(_p(f, ctypes.c_double), float(rho), float(ux), float(uy), float(uz))
    return f


def check_geometry3(p, solid):
    return _lib().ora3_check_geometry(ctypes.byref(p), _p(np.ascontiguousarray(solid, np.uint8), ctypes.c_uint8))


def inlet_profile3(p, solid):
    u = np.zeros((p.nz, p.ny))
    _lib().ora3_inlet_profile(ctypes.byref(p), _p(np.ascontiguousarray(solid, np.uint8), ctypes.c_uint8),
                              _p(u, ctypes.c_double))
    return u


def outlet_ids3(p, solid):
    ids = np.zeros((p.nz, p.ny), np.int32)
    n = _lib().ora3_outlet_ids(ctypes.byref(p), _p(np.ascontiguousarray(solid, np.uint8), ctypes.c_uint8),
                               _p(ids, ctypes.c_int32))
    return ids, n


def init3(p, solid):
    f = np.zeros((19,) + solid.shape)
    _lib().ora3_init(ctypes.byref(p), _p(np.ascontiguousarray(solid, np.uint8), ctypes.c_uint8),
                     _p(f, ctypes.c_double))
    return f


def init_state3(p, solid, rho, ux, uy, uz):
    f = np.zeros((19,) + solid.shape)
    arrs = [np.ascontiguousarray(a, np.float64) for a in (rho, ux, uy, uz)]
    _lib().ora3_init_state(ctypes.byref(p), _p(np.ascontiguousarray(solid, np.uint8), ctypes.c_uint8),
                           *[_p(a, ctypes.c_double) for a in arrs], _p(f, ctypes.c_double))
    return f


def run3(p, solid, u_in, f, n_steps):
    """Advance the post-collision state f (copied) by n_steps; returns (f, rho, ux, uy, uz, status)."""
    f = np.ascontiguousarray(f, np.float64).copy()
    work = np.empty_like(f)
    rho, ux, uy, uz = (np.zeros(solid.shape) for _ in range(4))
    st = _lib().ora3_run(ctypes.byref(p), _p(np.ascontiguousarray(solid, np.uint8), ctypes.c_uint8),
                         _p(np.ascontiguousarray(u_in, np.float64), ctypes.c_double), _p(f, ctypes.c_double),
                         _p(work, ctypes.c_double), int(n_steps), *[_p(a, ctypes.c_double) for a in (rho, ux, uy, uz)])
    return f, rho, ux, uy, uz, st


def observables3(p, solid, rho, ux, ids, n_out):
    dp, m_in = ctypes.c_double(), ctypes.c_double()
    m_out = np.zeros(max(1, n_out))
    _lib().ora3_observables(ctypes.byref(p), _p(np.ascontiguousarray(solid, np.uint8), ctypes.c_uint8),
                            _p(np.ascontiguousarray(rho), ctypes.c_double), _p(np.ascontiguousarray(ux), ctypes.c_double),
                            _p(np.ascontiguousarray(ids, np.int32), ctypes.c_int32), int(n_out), ctypes.byref(dp),
                            ctypes.byref(m_in), _p(m_out, ctypes.c_double))
    return dp.value, m_in.value, m_out[:n_out].copy()


def scores3(p, solid, rho, ux, uy, uz):
    cand = np.zeros(solid.shape, np.uint8)
    score = np.zeros(solid.shape)
    mu = p.rho0 * ((p.tau - 0.5) / 3.0)
    arrs = [np.ascontiguousarray(a, np.float64) for a in (rho, ux, uy, uz)]
    _lib().ora3_scores(ctypes.byref(p), _p(np.ascontiguousarray(solid, np.uint8), ctypes.c_uint8),
                       *[_p(a, ctypes.c_double) for a in arrs], float(mu), _p(cand, ctypes.c_uint8),
                       _p(score, ctypes.c_double))
    return cand, score


def select3(p, cand, score, n_swap):
    """The deterministic choice of Sec. 2.3 step 3 on the flat candidate arrays."""
    flat = make_params(int(cand.size), 1, p.tau)
    return select(flat, cand.reshape(-1), score.reshape(-1), n_swap)


def apply3(p, solid, f, fi, si, reinit=REINIT_WARM):
    return _lib().ora3_apply(ctypes.byref(p), _p(solid, ctypes.c_uint8), _p(f, ctypes.c_double),
                             _p(np.ascontiguousarray(fi, np.int32), ctypes.c_int32),
                             _p(np.ascontiguousarray(si, np.int32), ctypes.c_int32), len(fi), int(reinit))


class Solver3:
    """The loop of Sec. 2.3 on the D3Q19 oracle."""

    def __init__(self, params, cell_types, reinit=REINIT_WARM):
        self.params = params
        self.solid = np.ascontiguousarray(cell_types, np.uint8).copy()
        if check_geometry3(params, self.solid) != 0:
            raise ValueError("geometry rejected")
        self.u_in = inlet_profile3(params, self.solid)
        self.ids, self.n_out = outlet_ids3(params, self.solid)
        self.f = init3(params, self.solid)
        self.reinit = reinit
        self.rho = self.ux = self.uy = self.uz = None

    def solve(self, n_steps):
        f, rho, ux, uy, uz, st = run3(self.params, self.solid, self.u_in, self.f, n_steps)
        if st != 0:
            raise FloatingPointError("oracle diverged")
        self.f, self.rho, self.ux, self.uy, self.uz = f, rho, ux, uy, uz
        dp, m_in, m_out = observables3(self.params, self.solid, rho, ux, self.ids, self.n_out)
        return dict(dp=dp, m_in=m_in, m_out=m_out)

    def pick(self, n_swap, rho=None, ux=None, uy=None, uz=None):
        cand, score = scores3(self.params, self.solid, self.rho if rho is None else rho,
                              self.ux if ux is None else ux, self.uy if uy is None else uy,
                              self.uz if uz is None else uz)
        return select3(self.params, cand, score, n_swap)

    def optimize_step(self, n_swap, n_steps):
        fi, si = self.pick(n_swap)
        fluid = apply3(self.params, self.solid, self.f, fi, si, self.reinit)
        out = self.solve(n_steps)
        out.update(n_swapped=len(fi), fluid_count=fluid, fluid_idx=fi, solid_idx=si)
        return out
