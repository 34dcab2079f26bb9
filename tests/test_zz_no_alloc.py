"""The allocation-free entry point mm_step_static_scratch against the context-based path.

Some callers may not call cudaMalloc (a host framework that owns all device memory under a
fixed budget, plug-ins inside it, real-time loops that forbid allocation after start-up).  For
them the library steps caller-owned device buffers with its scratch in one static device array.
These tests call that entry point through the C ABI twice in a row, on two different problems
(the second with diffuse walls, so stale scratch from the first call would show), and compare
with mm_create / mm_set_state / mm_step / mm_get_* on the same inputs.  This file is collected
last so that a failure here cannot hide any other test's result.
"""
import numpy as np
import pytest

from helpers import q_rel_err
from paper_2509_21832_gb300 import api
from paper_2509_21832_gb300 import inputs as I


def _context_path(grid, params, Q, G, dt, eps, nsteps):
    with api.Solver(grid, params) as s:
        s.set_state(Q, G)
        s.step(dt, eps, nsteps)
        Qo, Ho = s.get_moments()
        Go = s.get_g()
    return Qo, Go, Ho


def _static_path(grid, params, Q, G, dt, eps, nsteps):
    import torch
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    Gd = torch.from_numpy(np.ascontiguousarray(G)).cuda()
    Hd = torch.full((4, grid.ny, grid.nx), float("nan"), dtype=torch.float64, device="cuda")
    api.mm_step_static_scratch(grid, params, Qd, Gd, Hd, dt, eps, nsteps,
                               stream=torch.cuda.current_stream().cuda_stream)
    return Qd.cpu().numpy(), Gd.cpu().numpy(), Hd.cpu().numpy()


@pytest.mark.gpu
def test_static_scratch_matches_context_path_two_calls():
    cases = [
        (I.Grid(nx=24, ny=20, nv1=24, nv2=24), I.Params(bc=(I.PERIODIC,) * 4), 0.05, 11),
        (I.Grid(nx=31, ny=17, nv1=16, nv2=20, v1min=-6, v1max=6, v2min=-6, v2max=6),
         I.Params(bc=(I.SPECULAR, I.EXTRAP, I.DIFFUSE, I.DIFFUSE), wall_T=(1.0, 1.0, 1.2, 0.9),
                  wall_U=(0.0, 0.0, 0.0, 0.15)), 0.01, 7),
    ]
    for grid, params, eps, nsteps in cases:
        Q = I.smooth_state(grid, seed=grid.nx, umax=0.2, aniso=0.05)
        G = I.seeded_g(grid, seed=grid.ny, amp=0.02)
        dt = api.mm_dt_for_cfl(grid, 0.5, 0.0, I.CFL_SUM)[0]
        Qa, Ga, Ha = _static_path(grid, params, Q, G, dt, eps, nsteps)
        Qb, Gb, Hb = _context_path(grid, params, Q, G, dt, eps, nsteps)
        assert np.all(q_rel_err(Qa, Qb) <= 1e-12)
        assert np.max(np.abs(Ga - Gb)) <= 1e-11 * np.max(np.abs(Gb))
        assert np.max(np.abs(Ha - Hb)) <= 1e-11 * np.max(np.abs(Hb))


def test_static_scratch_rejects_problems_beyond_its_limits():
    """Rejected before any device work, with a message naming the limit."""
    grid = I.Grid(nx=200, ny=100, nv1=8, nv2=8)   # 20000 cells > 16384
    with pytest.raises(api.MMError) as e:
        api.mm_step_static_scratch(grid, I.Params(), _Fake(6 * grid.ncell),
                                   _Fake(grid.nphase), _Fake(4 * grid.ncell), 1e-3, 0.1, 1)
    assert e.value.status == api.MM_ERR_INVALID_ARG and "too large" in str(e.value)
    grid = I.Grid(nx=40, ny=40, nv1=32, nv2=32)   # 1.6M phase cells > 1048576
    with pytest.raises(api.MMError) as e:
        api.mm_step_static_scratch(grid, I.Params(), _Fake(6 * grid.ncell),
                                   _Fake(grid.nphase), _Fake(4 * grid.ncell), 1e-3, 0.1, 1)
    assert e.value.status == api.MM_ERR_INVALID_ARG and "too large" in str(e.value)
    grid = I.Grid(nx=8, ny=8, nv1=8, nv2=8)
    with pytest.raises(api.MMError) as e:
        api.mm_step_static_scratch(grid, I.Params(precision=I.PREC_G_FP32), _Fake(6 * 64),
                                   _Fake(64 * 64), _Fake(4 * 64), 1e-3, 0.1, 1)
    assert e.value.status == api.MM_ERR_INVALID_ARG
    # buffers off the alignment that mm_create_borrowed asks for are refused, not stepped
    for q, g, h in ((4104, 4096, 4096), (4096, 4104, 4096), (4096, 4096, 4104), (4096, 4352 + 16, 4096)):
        with pytest.raises(api.MMError) as e:
            api.mm_step_static_scratch(grid, I.Params(), _Fake(6 * 64, q), _Fake(64 * 64, g),
                                       _Fake(4 * 64, h), 1e-3, 0.1, 1)
        assert e.value.status == api.MM_ERR_INVALID_ARG and "aligned" in str(e.value)


class _Fake:
    """Stand-in device tensor for argument checks that return before any device access."""

    is_cuda = True

    def __init__(self, n, ptr=4096):
        self.n = n
        self.ptr = ptr
        import torch
        self.dtype = torch.float64

    def element_size(self):
        return 8

    def is_contiguous(self):
        return True

    def numel(self):
        return self.n

    def data_ptr(self):
        return self.ptr
