"""Thin Python binding of libmmkfvs (include/mmkfvs.h): argument marshalling only.

Every step of the scheme runs in the CUDA library; this module only converts numpy arrays /
torch tensors to pointers.  The functions keep the C names (mm_create, mm_set_state, mm_step,
...); ``Solver`` wraps a context.  Importing this module on a machine without the built library
raises immediately: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

MM_OK, MM_ERR_INVALID_ARG, MM_ERR_OOM, MM_ERR_CUDA, MM_ERR_NONPHYSICAL, MM_ERR_TIMEOUT, \
    MM_ERR_STATE = range(7)
STATUS_NAMES = {0: "MM_OK", 1: "MM_ERR_INVALID_ARG", 2: "MM_ERR_OOM", 3: "MM_ERR_CUDA",
                4: "MM_ERR_NONPHYSICAL", 5: "MM_ERR_TIMEOUT", 6: "MM_ERR_STATE"}

_dp = ctypes.POINTER(ctypes.c_double)


class mm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("nv1", ctypes.c_int), ("nv2", ctypes.c_int),
                ("v1min", ctypes.c_double), ("v1max", ctypes.c_double),
                ("v2min", ctypes.c_double), ("v2max", ctypes.c_double)]


class mm_params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("tau_model", ctypes.c_int), ("tau0", ctypes.c_double),
                ("bc", ctypes.c_int * 4), ("wall_T", ctypes.c_double * 4),
                ("wall_U", ctypes.c_double * 4), ("wall_keep_es_term", ctypes.c_int),
                ("precision", ctypes.c_int)]


class mm1d_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("nv", ctypes.c_int), ("vmin", ctypes.c_double), ("vmax", ctypes.c_double)]


class mm1d_params(ctypes.Structure):
    _fields_ = [("bc", ctypes.c_int * 2), ("tau_model", ctypes.c_int), ("tau0", ctypes.c_double)]


TAU1D_HARDSPHERE, TAU1D_CONST = 0, 1


EXPORTS = ["mm_create", "mm_create_borrowed", "mm_scratch_bytes", "mm_device_bytes",
           "mm_set_state", "mm_set_state_device", "mm_set_state_prim", "mm_step",
           "mm_sync", "mm_get_moments", "mm_get_moments_device", "mm_get_g", "mm_dt_for_cfl",
           "mm_last_error", "mm_set_timing", "mm_get_timing", "mm_num_kernels",
           "mm_kernel_name", "mm_destroy", "mm_step_static_scratch", "mm_diag_exp", "mm_step_host",
           "mm_diag_erf", "mm_diag_bounded_wait", "mm_diag_fp64_fma",
           "mm_batch_create", "mm_batch_set_state", "mm_batch_step", "mm_batch_autotune",
           "mm_batch_set_graph", "mm_batch_sync", "mm_batch_get_moments", "mm_batch_get_g",
           "mm_batch_tiles", "mm_batch_diag_hold",
           "mm_batch_last_error", "mm_batch_destroy",
           "mm_mlp_create", "mm_mlp_set_params", "mm_mlp_get_params", "mm_mlp_forward",
           "mm_mlp_grad", "mm_mlp_train_step", "mm_mlp_last_error", "mm_mlp_destroy",
           "mm_set_closure", "mm_closure_features", "mm_closure_collect", "mm_closure_flags",
           "mm_closure_stats", "mm_set_closure_fallback", "mm_closure_steps",
           "mm_g_region_changed", "mm_mms_enable", "mm_mms_set_exact", "mm_mms_error",
           "mm1d_create", "mm1d_set_state", "mm1d_step", "mm1d_get_state", "mm1d_mms_enable",
           "mm1d_mms_set_exact", "mm1d_last_error", "mm1d_destroy"]

MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_NPARAM = 39, 64, 4, 6980

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libmmkfvs.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_needed else _build.LIB
    if not os.path.exists(path):
        raise ImportError("libmmkfvs.so is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    G, P = ctypes.POINTER(mm_grid), ctypes.POINTER(mm_params)
    vp = ctypes.c_void_p
    L.mm_create.argtypes = [G, P, vp, ctypes.POINTER(vp)]
    L.mm_device_bytes.argtypes = [G, P]
    L.mm_device_bytes.restype = ctypes.c_size_t
    L.mm_scratch_bytes.argtypes = [G, P]
    L.mm_scratch_bytes.restype = ctypes.c_size_t
    L.mm_create_borrowed.argtypes = [G, P, vp, vp, vp, vp, ctypes.c_size_t, ctypes.POINTER(vp)]
    L.mm_set_state_prim.argtypes = [vp, vp, vp, vp, vp]
    L.mm_set_state.argtypes = [vp, vp, vp]
    L.mm_set_state_device.argtypes = [vp, vp, vp]
    L.mm_step.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    L.mm_sync.argtypes = [vp]
    L.mm_get_moments.argtypes = [vp, vp, vp]
    L.mm_step_host.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, vp, vp]
    L.mm_get_moments_device.argtypes = [vp, vp, vp]
    L.mm_get_g.argtypes = [vp, vp]
    L.mm_dt_for_cfl.argtypes = [G, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_int)]
    L.mm_dt_for_cfl.restype = ctypes.c_double
    L.mm_last_error.argtypes = [vp]
    L.mm_last_error.restype = ctypes.c_char_p
    L.mm_set_timing.argtypes = [vp, ctypes.c_int]
    L.mm_get_timing.argtypes = [vp, _dp, ctypes.POINTER(ctypes.c_longlong)]
    L.mm_num_kernels.argtypes = []
    L.mm_num_kernels.restype = ctypes.c_int
    L.mm_kernel_name.argtypes = [ctypes.c_int]
    L.mm_kernel_name.restype = ctypes.c_char_p
    L.mm_destroy.argtypes = [vp]
    L.mm_destroy.restype = None
    L.mm_batch_create.argtypes = [ctypes.c_int, G, P, vp, ctypes.POINTER(vp)]
    L.mm_batch_set_state.argtypes = [vp, ctypes.c_int, vp, vp]
    L.mm_batch_step.argtypes = [vp, _dp, _dp, ctypes.c_int]
    L.mm_batch_autotune.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.mm_batch_set_graph.argtypes = [vp, ctypes.c_int]
    L.mm_batch_tiles.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.mm_batch_diag_hold.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double]
    L.mm_batch_sync.argtypes = [vp]
    L.mm_batch_get_moments.argtypes = [vp, ctypes.c_int, vp, vp]
    L.mm_batch_get_g.argtypes = [vp, ctypes.c_int, vp]
    L.mm_batch_last_error.argtypes = [vp]
    L.mm_batch_last_error.restype = ctypes.c_char_p
    L.mm_batch_destroy.argtypes = [vp]
    L.mm_batch_destroy.restype = None
    for name in ["mm_batch_create", "mm_batch_set_state", "mm_batch_step", "mm_batch_autotune",
                 "mm_batch_set_graph", "mm_batch_sync", "mm_batch_get_moments",
                 "mm_batch_get_g", "mm_batch_tiles", "mm_batch_diag_hold"]:
        getattr(L, name).restype = ctypes.c_int
    L.mm_diag_exp.argtypes = [vp, vp, vp, ctypes.c_size_t, vp]
    L.mm_diag_exp.restype = ctypes.c_int
    L.mm_diag_erf.argtypes = [vp, vp, vp, ctypes.c_size_t, vp]
    L.mm_diag_erf.restype = ctypes.c_int
    L.mm_diag_bounded_wait.argtypes = [ctypes.c_int, ctypes.c_int, vp]
    L.mm_diag_bounded_wait.restype = ctypes.c_int
    L.mm_diag_fp64_fma.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
    L.mm_diag_fp64_fma.restype = ctypes.c_int
    L.mm_step_static_scratch.argtypes = [G, P, vp, vp, vp, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, vp, ctypes.c_char_p, ctypes.c_size_t]
    L.mm_step_static_scratch.restype = ctypes.c_int
    fp = ctypes.POINTER(ctypes.c_float)
    L.mm_mlp_create.argtypes = [vp, ctypes.POINTER(vp)]
    L.mm_mlp_set_params.argtypes = [vp, fp, fp]
    L.mm_mlp_get_params.argtypes = [vp, fp, fp]
    L.mm_mlp_forward.argtypes = [vp, vp, vp, ctypes.c_int]
    L.mm_mlp_grad.argtypes = [vp, vp, vp, ctypes.c_int, fp, fp]
    L.mm_mlp_train_step.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_float, fp]
    L.mm_mlp_last_error.argtypes = [vp]
    L.mm_mlp_last_error.restype = ctypes.c_char_p
    L.mm_mlp_destroy.argtypes = [vp]
    L.mm_mlp_destroy.restype = None
    L.mm_set_closure.argtypes = [vp, vp, ctypes.c_double]
    L.mm_closure_features.argtypes = [vp, ctypes.c_double, ctypes.c_double, vp, vp]
    L.mm_closure_collect.argtypes = [vp, ctypes.c_double, ctypes.c_double, vp, vp]
    L.mm_closure_flags.argtypes = [vp, vp]
    L.mm_closure_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong),
                                   ctypes.POINTER(ctypes.c_longlong)]
    L.mm_set_closure_fallback.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    L.mm_g_region_changed.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.mm_closure_steps.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong),
                                   ctypes.POINTER(ctypes.c_longlong)]
    G1, P1 = ctypes.POINTER(mm1d_grid), ctypes.POINTER(mm1d_params)
    L.mm1d_create.argtypes = [G1, P1, vp, ctypes.POINTER(vp)]
    L.mm1d_set_state.argtypes = [vp, vp, vp]
    L.mm1d_step.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    L.mm1d_get_state.argtypes = [vp, vp, vp, vp]
    L.mm1d_mms_enable.argtypes = [vp, ctypes.c_int, ctypes.c_double]
    L.mm1d_mms_set_exact.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    L.mm1d_last_error.argtypes = [vp]
    L.mm1d_last_error.restype = ctypes.c_char_p
    L.mm1d_destroy.argtypes = [vp]
    L.mm1d_destroy.restype = None
    for name in ["mm1d_create", "mm1d_set_state", "mm1d_step", "mm1d_get_state",
                 "mm1d_mms_enable", "mm1d_mms_set_exact"]:
        getattr(L, name).restype = ctypes.c_int
    L.mm_mms_enable.argtypes = [vp, ctypes.c_int, ctypes.c_double]
    L.mm_mms_set_exact.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    L.mm_mms_error.argtypes = [vp, ctypes.c_double, ctypes.c_double, _dp, _dp]
    for name in ["mm_mms_enable", "mm_mms_set_exact", "mm_mms_error"]:
        getattr(L, name).restype = ctypes.c_int
    for name in ["mm_create", "mm_set_state", "mm_set_state_device", "mm_step", "mm_sync",
                 "mm_get_moments", "mm_get_moments_device", "mm_get_g", "mm_set_timing",
                 "mm_get_timing", "mm_mlp_create", "mm_mlp_set_params", "mm_mlp_get_params",
                 "mm_mlp_forward", "mm_mlp_grad", "mm_mlp_train_step", "mm_set_closure",
                 "mm_closure_features", "mm_closure_collect", "mm_closure_flags",
                 "mm_closure_stats", "mm_set_closure_fallback", "mm_closure_steps",
                 "mm_g_region_changed"]:
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class MMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def to_c_grid(g) -> mm_grid:
    return mm_grid(int(g.nx), int(g.ny), float(g.x0), float(g.x1), float(g.y0), float(g.y1),
                   int(g.nv1), int(g.nv2), float(g.v1min), float(g.v1max), float(g.v2min),
                   float(g.v2max))


def to_c_params(p) -> mm_params:
    o = mm_params()
    o.nu = float(p.nu)
    o.tau_model = int(p.tau_model)
    o.tau0 = float(p.tau0)
    for s in range(4):
        o.bc[s] = int(p.bc[s])
        o.wall_T[s] = float(p.wall_T[s])
        o.wall_U[s] = float(p.wall_U[s])
    o.wall_keep_es_term = int(p.wall_keep_es_term)
    o.precision = int(getattr(p, "precision", 0))
    return o


def _host_ptr(a, n):
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise TypeError("expected a C-contiguous float64 numpy array")
    if a.size != n:
        raise ValueError("host array has %d elements, expected %d" % (a.size, n))
    return a.ctypes.data


def _dev_ptr(t, n):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8):
        raise TypeError("expected a float64 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("device tensor must be contiguous")
    if t.numel() != n:
        raise ValueError("device tensor has %d elements, expected %d" % (t.numel(), n))
    return t.data_ptr()


# ---- the C entry points under their own names --------------------------------------------

def mm_dt_for_cfl(grid, cfl, t_final, form):
    n = ctypes.c_int(0)
    g = to_c_grid(grid)
    dt = load().mm_dt_for_cfl(ctypes.byref(g), float(cfl), float(t_final), int(form),
                              ctypes.byref(n))
    if dt < 0:
        raise MMError(MM_ERR_INVALID_ARG, "mm_dt_for_cfl")
    return dt, n.value


def mm_device_bytes(grid, params):
    g, p = to_c_grid(grid), to_c_params(params)
    return load().mm_device_bytes(ctypes.byref(g), ctypes.byref(p))


def mm_create(grid, params, stream=0):
    L = load()
    g, p = to_c_grid(grid), to_c_params(params)
    ctx = ctypes.c_void_p()
    st = L.mm_create(ctypes.byref(g), ctypes.byref(p), ctypes.c_void_p(int(stream)),
                     ctypes.byref(ctx))
    if st != MM_OK:
        raise MMError(st, "mm_create rejected the grid/parameters or could not allocate")
    return ctx


def mm_scratch_bytes(grid, params):
    g, p = to_c_grid(grid), to_c_params(params)
    return load().mm_scratch_bytes(ctypes.byref(g), ctypes.byref(p))


def mm_create_borrowed(grid, params, Q_ptr, G_ptr, scratch_ptr, scratch_bytes, stream=0):
    """A context on caller-owned device memory given as integer addresses (mm_create_borrowed);
    returns (status, ctx)."""
    L = load()
    g, p = to_c_grid(grid), to_c_params(params)
    ctx = ctypes.c_void_p()
    st = L.mm_create_borrowed(ctypes.byref(g), ctypes.byref(p), ctypes.c_void_p(int(stream)),
                              ctypes.c_void_p(int(Q_ptr)), ctypes.c_void_p(int(G_ptr)),
                              ctypes.c_void_p(int(scratch_ptr)), int(scratch_bytes),
                              ctypes.byref(ctx))
    return st, ctx


def mm_step_static_scratch(grid, params, Q_dev, G_dev, H_dev, dt, eps, nsteps, stream=0):
    """Advance nsteps steps in place on caller-owned FP64 CUDA tensors Q [6][ny][nx],
    G [ny][nx][nv2][nv1] and H [4][ny][nx] (output) without any device allocation: the scratch
    is one static device array of the library (size limits MM_STATIC_MAX_CELLS = 16384 cells
    and MM_STATIC_MAX_PHASE = 1048576 phase cells).  For callers that may not allocate device
    memory.  Calls that overlap on the GPU share that scratch and race."""
    ncell = grid.nx * grid.ny
    nphase = ncell * grid.nv1 * grid.nv2
    g, p = to_c_grid(grid), to_c_params(params)
    buf = ctypes.create_string_buffer(256)
    st = load().mm_step_static_scratch(ctypes.byref(g), ctypes.byref(p),
                                       _dev_ptr(Q_dev, 6 * ncell), _dev_ptr(G_dev, nphase),
                                       _dev_ptr(H_dev, 4 * ncell), float(dt), float(eps),
                                       int(nsteps), ctypes.c_void_p(int(stream)), buf, 256)
    if st != MM_OK:
        raise MMError(st, "mm_step_static_scratch: " + buf.value.decode())


def mm_diag_exp(x_dev, stream=0):
    """(fast, library) exponentials of a CUDA float64 tensor, computed on the device."""
    import torch
    yf, yl = torch.empty_like(x_dev), torch.empty_like(x_dev)
    st = load().mm_diag_exp(x_dev.data_ptr(), yf.data_ptr(), yl.data_ptr(), x_dev.numel(),
                            ctypes.c_void_p(int(stream)))
    if st != MM_OK:
        raise MMError(st, "mm_diag_exp")
    return yf, yl


def mm_diag_erf(x_dev, stream=0):
    """(flux, library) error functions of a CUDA float64 tensor, computed on the device."""
    import torch
    if not isinstance(x_dev, torch.Tensor) or not x_dev.is_cuda or x_dev.dtype != torch.float64:
        raise TypeError("expected a float64 CUDA tensor")
    x_dev = x_dev.contiguous()
    yf, yl = torch.empty_like(x_dev), torch.empty_like(x_dev)
    st = load().mm_diag_erf(x_dev.data_ptr(), yf.data_ptr(), yl.data_ptr(), x_dev.numel(),
                            ctypes.c_void_p(int(stream)))
    if st != MM_OK:
        raise MMError(st, "mm_diag_erf")
    return yf, yl


def mm_diag_fp64_fma(out_dev, ctas, iters, stream=0):
    """Launch the FP64 FMA probe (ctas x 256 threads, iters rounds of 8 chains) on stream without
    synchronising; out_dev is a float64 CUDA tensor of ctas * 256 elements.  Returns the flops."""
    _dev_ptr(out_dev, ctas * 256)
    st = load().mm_diag_fp64_fma(out_dev.data_ptr(), int(ctas), int(iters),
                                 ctypes.c_void_p(int(stream)))
    if st != MM_OK:
        raise MMError(st, "mm_diag_fp64_fma")
    return float(ctas) * 256 * iters * 16


def mm_diag_bounded_wait(copy, spins=1 << 16, stream=0):
    """Status of one bounded mbarrier wait on the device: MM_OK when the 16-byte bulk copy that
    completes it was issued (copy=True), MM_ERR_TIMEOUT when nothing completes it."""
    return load().mm_diag_bounded_wait(1 if copy else 0, int(spins), ctypes.c_void_p(int(stream)))


def _check(ctx, st, what):
    if st != MM_OK:
        raise MMError(st, "%s: %s" % (what, load().mm_last_error(ctx).decode()))


class Solver:
    """One device context: state (Q, G, H) of a problem on the GPU."""

    def __init__(self, grid, params, stream=0, borrow=None):
        """borrow = (Q, G, scratch): CUDA tensors that the context works in instead of its own
        allocations (mm_create_borrowed): Q float64 [6][ny][nx], G [ny][nx][nv2][nv1] float64 (or
        float32 for FP32 g), scratch a byte tensor of at least mm_scratch_bytes(grid, params);
        they must outlive the context."""
        self.grid, self.params = grid, params
        self.ncell = grid.nx * grid.ny
        self.nphase = self.ncell * grid.nv1 * grid.nv2
        self.L = load()
        self.borrow = borrow
        if borrow is None:
            self.ctx = mm_create(grid, params, stream)
        else:
            Q, G, S = borrow
            _dev_ptr(Q, 6 * self.ncell)
            gsize = 4 if int(getattr(params, "precision", 0)) == 1 else 8
            if not (G.is_cuda and G.is_contiguous() and G.numel() == self.nphase
                    and G.element_size() == gsize):
                raise ValueError("borrowed g must be a contiguous CUDA tensor of %d elements of "
                                 "%d bytes" % (self.nphase, gsize))
            if not (S.is_cuda and S.is_contiguous()):
                raise ValueError("borrowed scratch must be a contiguous CUDA tensor")
            st, ctx = mm_create_borrowed(grid, params, Q.data_ptr(), G.data_ptr(), S.data_ptr(),
                                         S.numel() * S.element_size(), stream)
            if st != MM_OK:
                raise MMError(st, "mm_create_borrowed rejected the grid/parameters or buffers")
            self.ctx = ctx

    def close(self):
        if self.ctx:
            self.L.mm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_state(self, Q, G=None):
        """Q [6][ny][nx] and G [ny][nx][nv2][nv1] (None: g = 0), numpy (host) or torch (cuda)."""
        if hasattr(Q, "is_cuda") and Q.is_cuda:
            st = self.L.mm_set_state_device(self.ctx, _dev_ptr(Q, 6 * self.ncell),
                                            _dev_ptr(G, self.nphase))
        else:
            Q = np.ascontiguousarray(Q, dtype=np.float64)
            G = None if G is None else np.ascontiguousarray(G, dtype=np.float64)
            st = self.L.mm_set_state(self.ctx, _host_ptr(Q, 6 * self.ncell),
                                     _host_ptr(G, self.nphase))
        _check(self.ctx, st, "mm_set_state")

    def set_state_prim(self, rho, u1, u2, T):
        """State from host primitive fields [ny][nx] with an isotropic temperature tensor and
        g = 0 (mm_set_state_prim)."""
        f = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, u1, u2, T)]
        st = self.L.mm_set_state_prim(self.ctx, *[_host_ptr(a, self.ncell) for a in f])
        _check(self.ctx, st, "mm_set_state_prim")

    def step(self, dt, eps, nsteps=1):
        _check(self.ctx, self.L.mm_step(self.ctx, float(dt), float(eps), int(nsteps)), "mm_step")

    def sync(self):
        _check(self.ctx, self.L.mm_sync(self.ctx), "mm_sync")

    def get_moments(self, Q_out=None, H_out=None, with_H=True):
        Q = Q_out if Q_out is not None else np.empty((6, self.grid.ny, self.grid.nx))
        H = H_out if H_out is not None else (
            np.empty((4, self.grid.ny, self.grid.nx)) if with_H else None)
        st = self.L.mm_get_moments(self.ctx, _host_ptr(Q, 6 * self.ncell),
                                   _host_ptr(H, 4 * self.ncell))
        _check(self.ctx, st, "mm_get_moments")
        return Q, H

    def step_host(self, Q, G, dt, eps, Q_out=None, H_out=None):
        """One step from host (Q, G) to host (Q^{n+1}, H): mm_step_host, the copy of G overlapped
        with the step (bitwise the result of set_state, step(dt, eps, 1), get_moments)."""
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        G = np.ascontiguousarray(G, dtype=np.float64)
        Qo = Q_out if Q_out is not None else np.empty((6, self.grid.ny, self.grid.nx))
        Ho = H_out if H_out is not None else np.empty((4, self.grid.ny, self.grid.nx))
        st = self.L.mm_step_host(self.ctx, _host_ptr(Q, 6 * self.ncell), _host_ptr(G, self.nphase),
                                 float(dt), float(eps), _host_ptr(Qo, 6 * self.ncell),
                                 _host_ptr(Ho, 4 * self.ncell))
        _check(self.ctx, st, "mm_step_host")
        return Qo, Ho

    def get_moments_device(self, Q_dev, H_dev=None):
        st = self.L.mm_get_moments_device(self.ctx, _dev_ptr(Q_dev, 6 * self.ncell),
                                          _dev_ptr(H_dev, 4 * self.ncell))
        _check(self.ctx, st, "mm_get_moments_device")

    def get_g(self):
        G = np.empty((self.grid.ny, self.grid.nx, self.grid.nv2, self.grid.nv1))
        _check(self.ctx, self.L.mm_get_g(self.ctx, _host_ptr(G, self.nphase)), "mm_get_g")
        return G

    def set_timing(self, enable=True):
        _check(self.ctx, self.L.mm_set_timing(self.ctx, int(enable)), "mm_set_timing")

    def get_timing(self):
        n = self.L.mm_num_kernels()
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        _check(self.ctx, self.L.mm_get_timing(self.ctx, ms, cnt), "mm_get_timing")
        return {self.L.mm_kernel_name(k).decode(): (ms[k], cnt[k]) for k in range(n)}

    def last_error(self):
        return self.L.mm_last_error(self.ctx).decode()

    # ---- manufactured-solution harness -------------------------------------------------------
    def mms_enable(self, enable=True, t0=0.0):
        _check(self.ctx, self.L.mm_mms_enable(self.ctx, int(enable), float(t0)), "mm_mms_enable")

    def mms_set_exact(self, t, eps):
        _check(self.ctx, self.L.mm_mms_set_exact(self.ctx, float(t), float(eps)), "mm_mms_set_exact")

    def mms_error(self, t, eps):
        """(macro, micro) relative L2 errors against the manufactured solution at time t."""
        a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(self.ctx, self.L.mm_mms_error(self.ctx, float(t), float(eps), ctypes.byref(a),
                                             ctypes.byref(b)), "mm_mms_error")
        return a.value, b.value

    # ---- learned closure -------------------------------------------------------------------
    def set_closure(self, mlp, threshold):
        """Hybrid stepping with the network mlp (an MLP, or None to switch it off)."""
        self._closure_mlp = mlp  # the context keeps the pointer: keep the network alive
        h = None if mlp is None else mlp.h
        _check(self.ctx, self.L.mm_set_closure(self.ctx, h, float(threshold)), "mm_set_closure")

    def closure_features(self, dt, eps, X_dev, aux_dev):
        """Features [nc][39] (float32 CUDA tensor) and [5][ny][nx] (float64: H_CE, scale)."""
        _check(self.ctx, self.L.mm_closure_features(self.ctx, float(dt), float(eps),
                                                   _f32_ptr(X_dev, self.ncell * MLP_IN),
                                                   _dev_ptr(aux_dev, 5 * self.ncell)),
               "mm_closure_features")

    def closure_collect(self, dt, eps, X_dev, Y_dev):
        """Features of Q^n, one plain step, targets (H - H_CE) / scale; float32 CUDA tensors."""
        _check(self.ctx, self.L.mm_closure_collect(self.ctx, float(dt), float(eps),
                                                  _f32_ptr(X_dev, self.ncell * MLP_IN),
                                                  _f32_ptr(Y_dev, self.ncell * MLP_OUT)),
               "mm_closure_collect")

    def closure_flags(self):
        f = np.zeros((self.grid.ny, self.grid.nx), dtype=np.uint8)
        _check(self.ctx, self.L.mm_closure_flags(self.ctx, f.ctypes.data), "mm_closure_flags")
        return f

    def closure_stats(self):
        a, b = ctypes.c_longlong(0), ctypes.c_longlong(0)
        _check(self.ctx, self.L.mm_closure_stats(self.ctx, ctypes.byref(a), ctypes.byref(b)),
               "mm_closure_stats")
        return a.value, b.value

    def g_region_changed(self, i0, i1, j0, j1):
        """g was changed by the caller in cells [i0, i1) x [j0, j1) (borrowed buffers)."""
        _check(self.ctx, self.L.mm_g_region_changed(self.ctx, int(i0), int(i1), int(j0),
                                                    int(j1)), "mm_g_region_changed")

    def set_closure_fallback(self, min_fraction, period):
        _check(self.ctx, self.L.mm_set_closure_fallback(self.ctx, float(min_fraction),
                                                        int(period)), "mm_set_closure_fallback")

    def closure_steps(self):
        """(hybrid steps, plain fallback steps) since the closure was set."""
        a, b = ctypes.c_longlong(0), ctypes.c_longlong(0)
        _check(self.ctx, self.L.mm_closure_steps(self.ctx, ctypes.byref(a), ctypes.byref(b)),
               "mm_closure_steps")
        return a.value, b.value


def _f32_ptr(t, n):
    if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 4):
        raise TypeError("expected a float32 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("device tensor must be contiguous")
    if t.numel() != n:
        raise ValueError("device tensor has %d elements, expected %d" % (t.numel(), n))
    return t.data_ptr()


def _host_f32(a, n):
    if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]):
        raise TypeError("expected a C-contiguous float32 numpy array")
    if a.size != n:
        raise ValueError("host array has %d elements, expected %d" % (a.size, n))
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class MLP:
    """The closure network (mm_mlp_*): BF16 weights, FP32 accumulation, trained on the GPU."""

    def __init__(self, params=None, norm=None, stream=0):
        self.L = load()
        self.h = ctypes.c_void_p()
        st = self.L.mm_mlp_create(ctypes.c_void_p(int(stream)), ctypes.byref(self.h))
        if st != MM_OK:
            raise MMError(st, "mm_mlp_create")
        if params is not None:
            self.set_params(params, norm)

    def _check(self, st, what):
        if st != MM_OK:
            raise MMError(st, "%s: %s" % (what, self.L.mm_mlp_last_error(self.h).decode()))

    def close(self):
        if self.h:
            self.L.mm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params, norm):
        p = np.ascontiguousarray(params, dtype=np.float32)
        n = np.ascontiguousarray(norm, dtype=np.float32)
        self._check(self.L.mm_mlp_set_params(self.h, _host_f32(p, MLP_NPARAM),
                                             _host_f32(n, 2 * MLP_IN + 2 * MLP_OUT)),
                    "mm_mlp_set_params")

    def get_params(self):
        """(FP32 master parameters, the BF16 parameters as FP32)."""
        a = np.zeros(MLP_NPARAM, dtype=np.float32)
        b = np.zeros(MLP_NPARAM, dtype=np.float32)
        self._check(self.L.mm_mlp_get_params(self.h, _host_f32(a, MLP_NPARAM),
                                             _host_f32(b, MLP_NPARAM)), "mm_mlp_get_params")
        return a, b

    def forward(self, X_dev, Y_dev):
        n = X_dev.shape[0]
        self._check(self.L.mm_mlp_forward(self.h, _f32_ptr(X_dev, n * MLP_IN),
                                          _f32_ptr(Y_dev, n * MLP_OUT), n), "mm_mlp_forward")

    def grad(self, X_dev, T_dev):
        """(loss, gradient) of the mean squared error of the standardised outputs."""
        n = X_dev.shape[0]
        g = np.zeros(MLP_NPARAM, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        self._check(self.L.mm_mlp_grad(self.h, _f32_ptr(X_dev, n * MLP_IN),
                                       _f32_ptr(T_dev, n * MLP_OUT), n, _host_f32(g, MLP_NPARAM),
                                       _host_f32(loss, 1)), "mm_mlp_grad")
        return float(loss[0]), g

    def train_step(self, X_dev, T_dev, lr, want_loss=False):
        n = X_dev.shape[0]
        loss = np.zeros(1, dtype=np.float32)
        self._check(self.L.mm_mlp_train_step(self.h, _f32_ptr(X_dev, n * MLP_IN),
                                             _f32_ptr(T_dev, n * MLP_OUT), n, float(lr),
                                             _host_f32(loss, 1) if want_loss else None),
                    "mm_mlp_train_step")
        return float(loss[0]) if want_loss else None


class Solver1D:
    """The 1D-1V BGK micro-macro scheme (mm1d_*)."""

    def __init__(self, nx, nv, x0=0.0, x1=1.0, vmin=-6.5, vmax=6.5, bc=(0, 0),
                 tau_model=TAU1D_HARDSPHERE, tau0=1.0, stream=0):
        self.nx, self.nv = nx, nv
        self.L = load()
        g = mm1d_grid(int(nx), float(x0), float(x1), int(nv), float(vmin), float(vmax))
        p = mm1d_params((ctypes.c_int * 2)(*bc), int(tau_model), float(tau0))
        self.ctx = ctypes.c_void_p()
        st = self.L.mm1d_create(ctypes.byref(g), ctypes.byref(p), ctypes.c_void_p(int(stream)),
                                ctypes.byref(self.ctx))
        if st != MM_OK:
            raise MMError(st, "mm1d_create rejected the grid/parameters or could not allocate")

    def _check(self, st, what):
        if st != MM_OK:
            raise MMError(st, "%s: %s" % (what, self.L.mm1d_last_error(self.ctx).decode()))

    def close(self):
        if self.ctx:
            self.L.mm1d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_state(self, Q, G=None):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        G = None if G is None else np.ascontiguousarray(G, dtype=np.float64)
        self._check(self.L.mm1d_set_state(self.ctx, _host_ptr(Q, 3 * self.nx),
                                          _host_ptr(G, self.nx * self.nv)), "mm1d_set_state")

    def step(self, dt, eps, nsteps=1):
        self._check(self.L.mm1d_step(self.ctx, float(dt), float(eps), int(nsteps)), "mm1d_step")

    def get_state(self):
        Q = np.empty((3, self.nx))
        G = np.empty((self.nx, self.nv))
        H = np.empty(self.nx)
        self._check(self.L.mm1d_get_state(self.ctx, Q.ctypes.data, G.ctypes.data, H.ctypes.data),
                    "mm1d_get_state")
        return Q, G, H

    def mms_enable(self, enable=True, t0=0.0):
        self._check(self.L.mm1d_mms_enable(self.ctx, int(enable), float(t0)), "mm1d_mms_enable")

    def mms_set_exact(self, t, eps):
        self._check(self.L.mm1d_mms_set_exact(self.ctx, float(t), float(eps)), "mm1d_mms_set_exact")


class BatchSolver:
    """Many independent problems stepped together (mm_batch_*)."""

    def __init__(self, grids, params, stream=0):
        self.L = load()
        self.grids, self.params = list(grids), list(params)
        n = len(self.grids)
        G = (mm_grid * n)(*[to_c_grid(g) for g in self.grids])
        P = (mm_params * n)(*[to_c_params(p) for p in self.params])
        self.b = ctypes.c_void_p()
        st = self.L.mm_batch_create(n, G, P, ctypes.c_void_p(int(stream)), ctypes.byref(self.b))
        if st != MM_OK:
            raise MMError(st, "mm_batch_create rejected the problems or could not allocate")
        self.n = n

    def _check(self, st, what):
        if st != MM_OK:
            raise MMError(st, "%s: %s" % (what, self.L.mm_batch_last_error(self.b).decode()))

    def close(self):
        if self.b:
            self.L.mm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_state(self, q, Q, G=None):
        g = self.grids[q]
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        G = None if G is None else np.ascontiguousarray(G, dtype=np.float64)
        st = self.L.mm_batch_set_state(self.b, int(q), _host_ptr(Q, 6 * g.nx * g.ny),
                                       _host_ptr(G, g.nx * g.ny * g.nv1 * g.nv2))
        self._check(st, "mm_batch_set_state")

    def step(self, dt, eps, nsteps=1):
        dt = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, float), (self.n,)))
        eps = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, float), (self.n,)))
        st = self.L.mm_batch_step(self.b, dt.ctypes.data_as(_dp), eps.ctypes.data_as(_dp),
                                  int(nsteps))
        self._check(st, "mm_batch_step")

    def autotune(self):
        t, c = ctypes.c_int(0), ctypes.c_int(0)
        self._check(self.L.mm_batch_autotune(self.b, ctypes.byref(t), ctypes.byref(c)),
                    "mm_batch_autotune")
        return t.value, c.value

    def set_graph(self, enable):
        self._check(self.L.mm_batch_set_graph(self.b, int(enable)), "mm_batch_set_graph")

    def tiles(self):
        """(cells per item of the phase-space phases, cells per item of the per-cell phases)."""
        a, c = ctypes.c_int(0), ctypes.c_int(0)
        self._check(self.L.mm_batch_tiles(self.b, ctypes.byref(a), ctypes.byref(c)),
                    "mm_batch_tiles")
        return a.value, c.value

    def diag_hold(self, q, phase, wait_ms=50.0):
        self._check(self.L.mm_batch_diag_hold(self.b, int(q), int(phase), float(wait_ms)),
                    "mm_batch_diag_hold")

    def sync(self):
        self._check(self.L.mm_batch_sync(self.b), "mm_batch_sync")

    def get_moments(self, q):
        g = self.grids[q]
        Q = np.empty((6, g.ny, g.nx))
        H = np.empty((4, g.ny, g.nx))
        self._check(self.L.mm_batch_get_moments(self.b, int(q), Q.ctypes.data, H.ctypes.data),
                    "mm_batch_get_moments")
        return Q, H

    def get_g(self, q):
        g = self.grids[q]
        G = np.empty((g.ny, g.nx, g.nv2, g.nv1))
        self._check(self.L.mm_batch_get_g(self.b, int(q), G.ctypes.data), "mm_batch_get_g")
        return G
