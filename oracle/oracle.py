"""ctypes wrapper of the plain FP64 CPU oracle (oracle/liboracle.so).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the CPU-baseline leg of
the benchmark.  It takes grid/parameter objects by duck typing (attributes nx, ny, x0, ...,
nu, tau_model, tau0, bc, wall_T, wall_U, wall_keep_es_term) and numpy arrays in the layouts
Q[6][ny][nx], G[ny][nx][nv2][nv1], H[4][ny][nx].
"""
import ctypes

import numpy as np

from . import build as _build

_c_double_p = ctypes.POINTER(ctypes.c_double)


class OrcGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("nv1", ctypes.c_int), ("nv2", ctypes.c_int),
                ("v1min", ctypes.c_double), ("v1max", ctypes.c_double),
                ("v2min", ctypes.c_double), ("v2max", ctypes.c_double)]


class OrcParams(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("tau_model", ctypes.c_int), ("tau0", ctypes.c_double),
                ("bc", ctypes.c_int * 4), ("wall_T", ctypes.c_double * 4),
                ("wall_U", ctypes.c_double * 4), ("wall_keep_es_term", ctypes.c_int)]


class Orc1dGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("nv", ctypes.c_int), ("vmin", ctypes.c_double), ("vmax", ctypes.c_double)]


class Orc1dParams(ctypes.Structure):
    _fields_ = [("bc", ctypes.c_int * 2), ("tau_model", ctypes.c_int), ("tau0", ctypes.c_double)]


TAU1D_HARDSPHERE, TAU1D_CONST = 0, 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(_build.build()))
    return _lib


class use_library:
    """Context manager: route every call of this module to another build of the oracle (a copy
    of its source with a planted mistake, built by build.build_variant) while the block runs."""

    def __init__(self, path):
        self.L = _configure(ctypes.CDLL(path))

    def __enter__(self):
        global _lib
        self.saved, _lib = _lib, self.L
        return self.L

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _configure(L):
    G, P = ctypes.POINTER(OrcGrid), ctypes.POINTER(OrcParams)
    L.orc_step.argtypes = [G, P, _c_double_p, _c_double_p, _c_double_p,
                           ctypes.c_double, ctypes.c_double, ctypes.c_int]
    L.orc_step.restype = ctypes.c_int
    L.orc_dt_for_cfl.argtypes = [G, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_int)]
    L.orc_dt_for_cfl.restype = ctypes.c_double
    L.orc_prims.argtypes = [P, _c_double_p, _c_double_p]
    L.orc_prims.restype = ctypes.c_int
    L.orc_q_from_prim.argtypes = [ctypes.c_int] + [_c_double_p] * 5
    L.orc_q_from_prim.restype = ctypes.c_int
    L.orc_maxwellian_gauss.argtypes = [P, _c_double_p, ctypes.c_double, ctypes.c_double,
                                       _c_double_p, _c_double_p]
    L.orc_maxwellian_gauss.restype = None
    L.orc_project.argtypes = [G, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double, _c_double_p, _c_double_p]
    L.orc_project.restype = None
    L.orc_kfvs_half.argtypes = [_c_double_p, ctypes.c_int, _c_double_p, _c_double_p]
    L.orc_kfvs_half.restype = None
    L.orc_wall_R.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    L.orc_wall_R.restype = ctypes.c_double
    L.orc_trbdf2_W.argtypes = [ctypes.c_double] * 4
    L.orc_trbdf2_W.restype = ctypes.c_double
    L.orc_step_closure.argtypes = [G, P, _c_double_p, _c_double_p, _c_double_p,
                                   ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_ubyte),
                                   ctypes.POINTER(ctypes.c_ubyte), _c_double_p]
    L.orc_step_closure.restype = ctypes.c_int
    L.orc_step_mms.argtypes = [G, P, _c_double_p, _c_double_p, _c_double_p,
                               ctypes.c_double, ctypes.c_double, ctypes.c_int,
                               ctypes.c_double]
    L.orc_step_mms.restype = ctypes.c_int
    L.orc_mms_exact.argtypes = [G, P, ctypes.c_double, ctypes.c_double, _c_double_p,
                                _c_double_p]
    L.orc_mms_exact.restype = ctypes.c_int
    L.orc_mms_source.argtypes = [G, P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, _c_double_p]
    L.orc_mms_source.restype = ctypes.c_int
    G1, P1 = ctypes.POINTER(Orc1dGrid), ctypes.POINTER(Orc1dParams)
    L.orc1d_step.argtypes = [G1, P1, _c_double_p, _c_double_p, _c_double_p, ctypes.c_double,
                             ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double]
    L.orc1d_step.restype = ctypes.c_int
    L.orc1d_mms_exact.argtypes = [G1, ctypes.c_double, ctypes.c_double, _c_double_p,
                                  _c_double_p]
    L.orc1d_mms_exact.restype = ctypes.c_int
    L.orc1d_dt.argtypes = [G1, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
    L.orc1d_dt.restype = ctypes.c_double
    L.orc_ghat.argtypes = [G, P, _c_double_p, ctypes.c_double, _c_double_p]
    L.orc_ghat.restype = ctypes.c_int
    L.orc_num_threads.argtypes = []
    L.orc_num_threads.restype = ctypes.c_int
    return L


def _grid(g) -> OrcGrid:
    return OrcGrid(int(g.nx), int(g.ny), float(g.x0), float(g.x1), float(g.y0), float(g.y1),
                   int(g.nv1), int(g.nv2), float(g.v1min), float(g.v1max),
                   float(g.v2min), float(g.v2max))


def _params(p) -> OrcParams:
    o = OrcParams()
    o.nu = float(p.nu)
    o.tau_model = int(p.tau_model)
    o.tau0 = float(p.tau0)
    for s in range(4):
        o.bc[s] = int(p.bc[s])
        o.wall_T[s] = float(p.wall_T[s])
        o.wall_U[s] = float(p.wall_U[s])
    o.wall_keep_es_term = int(p.wall_keep_es_term)
    return o


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_c_double_p)


class OracleError(RuntimeError):
    pass


def step(grid, params, Q, G, dt, eps, nsteps=1):
    """Return (Q, G, H) after nsteps steps; inputs are not modified."""
    Q = np.array(Q, dtype=np.float64, order="C", copy=True)
    G = np.array(G, dtype=np.float64, order="C", copy=True)
    H = np.zeros((4, grid.ny, grid.nx), dtype=np.float64)
    assert Q.size == 6 * grid.nx * grid.ny
    assert G.size == grid.nx * grid.ny * grid.nv1 * grid.nv2
    gg, pp = _grid(grid), _params(params)
    rc = lib().orc_step(ctypes.byref(gg), ctypes.byref(pp), _ptr(Q), _ptr(G), _ptr(H),
                        float(dt), float(eps), int(nsteps))
    if rc != 0:
        raise OracleError("orc_step returned %d" % rc)
    return Q, G, H


def step_closure(grid, params, Q, G, dt, eps, closure, refresh, Hcl):
    """One hybrid step: cells with refresh != 0 first take g^n = Ghat(Q^n); cells with
    closure != 0 then keep g^n and feed the heat flux Hcl [4][ny][nx] to the macro step; returns
    (Q, G, H).  Inputs are not modified."""
    Q = np.array(Q, dtype=np.float64, order="C", copy=True)
    G = np.array(G, dtype=np.float64, order="C", copy=True)
    H = np.zeros((4, grid.ny, grid.nx), dtype=np.float64)
    fl = np.ascontiguousarray(np.asarray(closure).reshape(-1) != 0, dtype=np.uint8)
    rf = np.ascontiguousarray(np.asarray(refresh).reshape(-1) != 0, dtype=np.uint8)
    assert rf.size == fl.size
    Hc = np.ascontiguousarray(Hcl, dtype=np.float64).reshape(4, grid.ny, grid.nx)
    assert fl.size == grid.nx * grid.ny
    gg, pp = _grid(grid), _params(params)
    rc = lib().orc_step_closure(ctypes.byref(gg), ctypes.byref(pp), _ptr(Q), _ptr(G), _ptr(H),
                                float(dt), float(eps),
                                fl.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                                rf.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), _ptr(Hc))
    if rc != 0:
        raise OracleError("orc_step_closure returned %d" % rc)
    return Q, G, H


def step_mms(grid, params, Q, G, dt, eps, nsteps, t0=0.0):
    """nsteps steps of the manufactured-solution problem from time t0; returns (Q, G, H)."""
    Q = np.array(Q, dtype=np.float64, order="C", copy=True)
    G = np.array(G, dtype=np.float64, order="C", copy=True)
    H = np.zeros((4, grid.ny, grid.nx), dtype=np.float64)
    gg, pp = _grid(grid), _params(params)
    rc = lib().orc_step_mms(ctypes.byref(gg), ctypes.byref(pp), _ptr(Q), _ptr(G), _ptr(H),
                            float(dt), float(eps), int(nsteps), float(t0))
    if rc != 0:
        raise OracleError("orc_step_mms returned %d" % rc)
    return Q, G, H


def mms_exact(grid, params, t, eps):
    """Exact (Q [6][ny][nx], g [ny][nx][nv2][nv1]) of the manufactured solution at time t."""
    Q = np.zeros((6, grid.ny, grid.nx))
    G = np.zeros((grid.ny, grid.nx, grid.nv2, grid.nv1))
    gg, pp = _grid(grid), _params(params)
    rc = lib().orc_mms_exact(ctypes.byref(gg), ctypes.byref(pp), float(t), float(eps), _ptr(Q),
                             _ptr(G))
    if rc != 0:
        raise OracleError("orc_mms_exact returned %d" % rc)
    return Q, G


def mms_source(grid, params, eps, t, x, y):
    """The manufactured residual S [nv2][nv1] at the point (x, y), time t."""
    S = np.zeros((grid.nv2, grid.nv1))
    gg, pp = _grid(grid), _params(params)
    rc = lib().orc_mms_source(ctypes.byref(gg), ctypes.byref(pp), float(eps), float(t),
                              float(x), float(y), _ptr(S))
    if rc != 0:
        raise OracleError("orc_mms_source returned %d" % rc)
    return S


def _g1(nx, nv, x0, x1, vmin, vmax):
    return Orc1dGrid(int(nx), float(x0), float(x1), int(nv), float(vmin), float(vmax))


def step1d(nx, nv, Q, G, dt, eps, nsteps, bc=(0, 0), tau_model=TAU1D_HARDSPHERE, tau0=1.0,
           x0=0.0, x1=1.0, vmin=-6.5, vmax=6.5, mms=False, t0=0.0):
    """1D-1V BGK micro-macro steps; returns (Q [3][nx], G [nx][nv], H [nx])."""
    Q = np.array(Q, dtype=np.float64, order="C", copy=True)
    G = np.array(G, dtype=np.float64, order="C", copy=True)
    H = np.zeros(nx)
    g = _g1(nx, nv, x0, x1, vmin, vmax)
    p = Orc1dParams((ctypes.c_int * 2)(*bc), int(tau_model), float(tau0))
    rc = lib().orc1d_step(ctypes.byref(g), ctypes.byref(p), _ptr(Q), _ptr(G), _ptr(H),
                          float(dt), float(eps), int(nsteps), int(bool(mms)), float(t0))
    if rc != 0:
        raise OracleError("orc1d_step returned %d" % rc)
    return Q, G, H


def mms1d_exact(nx, nv, t, eps, x0=0.0, x1=1.0, vmin=-6.5, vmax=6.5):
    Q = np.zeros((3, nx))
    G = np.zeros((nx, nv))
    g = _g1(nx, nv, x0, x1, vmin, vmax)
    rc = lib().orc1d_mms_exact(ctypes.byref(g), float(t), float(eps), _ptr(Q), _ptr(G))
    if rc != 0:
        raise OracleError("orc1d_mms_exact returned %d" % rc)
    return Q, G


def dt1d(nx, nv, cfl, t_final, x0=0.0, x1=1.0, vmin=-6.5, vmax=6.5):
    n = ctypes.c_int(0)
    g = _g1(nx, nv, x0, x1, vmin, vmax)
    dt = lib().orc1d_dt(ctypes.byref(g), float(cfl), float(t_final), ctypes.byref(n))
    return dt, n.value


def dt_for_cfl(grid, cfl, t_final, form):
    n = ctypes.c_int(0)
    gg = _grid(grid)
    dt = lib().orc_dt_for_cfl(ctypes.byref(gg), float(cfl), float(t_final), int(form),
                              ctypes.byref(n))
    return dt, n.value


def q_from_prim(rho, u1, u2, T):
    """Q [6][...] from primitive fields of equal shape with an isotropic temperature tensor
    (orc_q_from_prim)."""
    fields = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, u1, u2, T)]
    shape = fields[0].shape
    if any(f.shape != shape for f in fields):
        raise ValueError("rho, u1, u2, T must have the same shape")
    n = int(np.prod(shape))
    Q = np.zeros((6,) + shape)
    if lib().orc_q_from_prim(n, *[_ptr(f) for f in fields], _ptr(Q)):
        raise OracleError("non-physical primitive state")
    return Q


def prims(params, q):
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(8)
    pp = _params(params)
    rc = lib().orc_prims(ctypes.byref(pp), _ptr(q), _ptr(out))
    if rc:
        raise OracleError("non-physical state")
    return out


def maxwellian_gauss(params, q, v1, v2):
    q = np.ascontiguousarray(q, dtype=np.float64)
    m, g = ctypes.c_double(), ctypes.c_double()
    pp = _params(params)
    lib().orc_maxwellian_gauss(ctypes.byref(pp), _ptr(q), float(v1), float(v2),
                               ctypes.byref(m), ctypes.byref(g))
    return m.value, g.value


def project(grid, rho, u1, u2, T, F):
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros_like(F)
    gg = _grid(grid)
    lib().orc_project(ctypes.byref(gg), float(rho), float(u1), float(u2), float(T),
                      _ptr(F), _ptr(out))
    return out


def kfvs_half(q, direction):
    q = np.ascontiguousarray(q, dtype=np.float64)
    Fp, Fm = np.zeros(6), np.zeros(6)
    lib().orc_kfvs_half(_ptr(q), int(direction), _ptr(Fp), _ptr(Fm))
    return Fp, Fm


def wall_R(ua, Taa, Tw, sign):
    return lib().orc_wall_R(float(ua), float(Taa), float(Tw), int(sign))


def trbdf2_W(tau, nu, eps, dt):
    return lib().orc_trbdf2_W(float(tau), float(nu), float(eps), float(dt))


def ghat(grid, params, Q, eps):
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    out = np.zeros((grid.ny, grid.nx, grid.nv2, grid.nv1))
    gg, pp = _grid(grid), _params(params)
    rc = lib().orc_ghat(ctypes.byref(gg), ctypes.byref(pp), _ptr(Q), float(eps), _ptr(out))
    if rc:
        raise OracleError("orc_ghat returned %d" % rc)
    return out


def num_threads():
    return lib().orc_num_threads()
