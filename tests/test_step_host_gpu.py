"""mm_step_host: one step from host state to host moments with the copy of g overlapped with the
micro sweeps (row chunks on a second stream) gives the result of mm_set_state + mm_step(1) +
mm_get_moments, for every chunking case: periodic y (the first chunk's y sweep deferred), rows
not divisible by the chunk count, fewer rows than chunks, diffuse walls, and the contexts that
run the calls in sequence (FP32 g).  Bit for bit where the mesh keeps no row sums (16^2, FP32 g);
to rounding (1e-13) where mm_step takes the x-sweep moments from them (32^2, 24^2)."""
import numpy as np
import pytest

from paper_2509_21832_gb300 import api
from paper_2509_21832_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = [
    ("specular_32", dict(nx=20, ny=37, nv1=32, nv2=32), (I.SPECULAR,) * 4, {}, I.PREC_FP64),
    ("periodic_24", dict(nx=13, ny=40, nv1=24, nv2=24), (I.PERIODIC,) * 4, {}, I.PREC_FP64),
    ("periodic_few_rows", dict(nx=11, ny=5, nv1=16, nv2=16), (I.PERIODIC,) * 4, {}, I.PREC_FP64),
    ("diffuse_16", dict(nx=12, ny=19, nv1=16, nv2=16), (I.EXTRAP, I.EXTRAP, I.DIFFUSE, I.DIFFUSE),
     dict(wall_T=(1.0, 1.0, 1.2, 0.9)), I.PREC_FP64),
    ("fp32_24", dict(nx=9, ny=18, nv1=24, nv2=24), (I.SPECULAR,) * 4, {}, I.PREC_G_FP32),
]


@pytest.mark.parametrize("name,gk,bc,extra,prec", CASES, ids=[c[0] for c in CASES])
def test_step_host_is_bitwise_the_three_calls(name, gk, bc, extra, prec):
    grid = I.Grid(**gk)
    params = I.Params(bc=bc, precision=prec, **extra)
    Q = I.smooth_state(grid, seed=len(name), umax=0.25, aniso=0.06)
    G = I.seeded_g(grid, seed=9, amp=0.02)
    dt = 0.4 / (8.0 * grid.nx + 8.0 * grid.ny)
    eps = 1e-2
    with api.Solver(grid, params) as s:
        s.set_state(Q, G)
        s.step(dt, eps, 1)
        Q1, H1 = s.get_moments()
        G1 = s.get_g()
    with api.Solver(grid, params) as s:
        Qw = np.zeros_like(Q1)  # a different prior state, overwritten by the call
        s.set_state(Qw + Q, None)
        s.step(dt, eps, 1)
        Q2, H2 = s.step_host(Q, G, dt, eps)
        G2 = s.get_g()
        # and again from the result, as a host-resident time loop does
        Q3, H3 = s.step_host(Q2, G2, dt, eps)
    with api.Solver(grid, params) as s:
        s.set_state(Q, G)
        s.step(dt, eps, 2)
        Q4, H4 = s.get_moments()

    def same(a, b):
        if grid.nv1 <= 16 or prec == I.PREC_G_FP32:
            return np.array_equal(a, b)
        return np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))

    assert same(Q1, Q2) and same(H1, H2) and same(G1, G2), name
    assert same(Q3, Q4) and same(H3, H4), name


def test_step_host_rejects_missing_buffers():
    grid = I.Grid(nx=8, ny=8, nv1=8, nv2=8)
    with api.Solver(grid, I.Params()) as s:
        st = s.L.mm_step_host(s.ctx, None, None, 1e-3, 1e-2, None, None)
        assert st == api.MM_ERR_INVALID_ARG


def test_step_host_full_size_benchmark_workload():
    """The benchmark's end-to-end path at full size (256^2 x 32^2 bump, specular walls: 18 ramped
    row chunks, y sweeps on two streams) against mm_set_state + mm_step + mm_get_moments: equal
    to rounding (the x sweep sums per velocity here, from row sums there), twice in a row."""
    pr = I.bump_specular(n=256, nv=32, eps=0.1, seed=0)
    G = I.seeded_g(pr.grid, seed=5, amp=0.02)
    with api.Solver(pr.grid, pr.params) as s:
        s.set_state(pr.Q, G)
        s.step(pr.dt, pr.eps, 1)
        Q1, H1 = s.get_moments()
        G1 = s.get_g()
        s.step(pr.dt, pr.eps, 1)
        Q2, H2 = s.get_moments()
    with api.Solver(pr.grid, pr.params) as s:
        s.set_state(pr.Q, None)
        Qa, Ha = s.step_host(pr.Q, G, pr.dt, pr.eps)
        Ga = s.get_g()
        Qb, Hb = s.step_host(Qa, Ga, pr.dt, pr.eps)

    def close(a, b):
        return np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))

    assert close(Qa, Q1) and close(Ha, H1) and close(Ga, G1)
    assert close(Qb, Q2) and close(Hb, H2)
