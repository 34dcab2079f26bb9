"""Bounded device waits: the FP32-g kernels wait on an mbarrier for their bulk copies, and every
such wait gives up after a fixed number of attempts with an error status instead of hanging.  The
diagnostic entry point runs the same wait with and without the copy that completes it; the
timed-out wait must come back as MM_ERR_TIMEOUT and leave the device usable."""
import numpy as np
import pytest

from paper_2509_21832_gb300 import api
from paper_2509_21832_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _fp32_run(grid, params, Q, G, dt, eps, n):
    with api.Solver(grid, params) as s:
        s.set_state(Q, G)
        s.step(dt, eps, n)
        Qg, Hg = s.get_moments()
        return Qg, Hg, s.get_g()


def test_wait_completes_with_its_copy():
    assert api.mm_diag_bounded_wait(True) == api.MM_OK


def test_wait_without_its_copy_times_out_and_the_device_stays_usable():
    grid = I.Grid(nx=9, ny=8, nv1=24, nv2=24)  # 24^2, symmetric: the staged kernel
    params = I.Params(bc=(I.SPECULAR,) * 4, precision=I.PREC_G_FP32)
    Q = I.smooth_state(grid, seed=5, umax=0.2, aniso=0.05)
    G = I.seeded_g(grid, seed=6, amp=0.02)
    dt, eps = 2e-3, 1e-2
    before = _fp32_run(grid, params, Q, G, dt, eps, 3)
    assert api.mm_diag_bounded_wait(False, spins=1 << 12) == api.MM_ERR_TIMEOUT
    assert api.mm_diag_bounded_wait(True) == api.MM_OK
    after = _fp32_run(grid, params, Q, G, dt, eps, 3)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)


def test_wait_rejects_a_nonpositive_limit():
    assert api.mm_diag_bounded_wait(True, spins=0) == api.MM_ERR_INVALID_ARG
