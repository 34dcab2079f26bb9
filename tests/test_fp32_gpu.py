"""FP32-g mixed precision (g stored and transported in FP32; projection coefficients, heat
flux totals and the macro update in FP64) against the FP64 oracle and the FP64 GPU path."""
import numpy as np
import pytest

from helpers import q_rel_err
from oracle import oracle as O
from paper_2509_21832_gb300 import api
from paper_2509_21832_gb300 import inputs as I

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24  # unit roundoff of FP32


def run(grid, params, Q, G, dt, eps, n):
    with api.Solver(grid, params) as s:
        s.set_state(Q, G)
        s.step(dt, eps, n)
        Qg, Hg = s.get_moments()
        Gg = s.get_g()
    return Qg, Gg, Hg


CASES = [
    ("periodic_24", dict(nx=13, ny=11, nv1=24, nv2=24), (I.PERIODIC,) * 4, {}),
    ("specular_32", dict(nx=10, ny=7, nv1=32, nv2=32), (I.SPECULAR,) * 4, {}),
    ("mixed_diffuse_16", dict(nx=12, ny=9, nv1=16, nv2=16),
     (I.EXTRAP, I.EXTRAP, I.DIFFUSE, I.EXTRAP), dict(wall_T=(1.0, 1.0, 1.1, 1.0))),
    ("odd_17x15", dict(nx=6, ny=5, nv1=17, nv2=15, v1min=-6, v1max=6, v2min=-6, v2max=6),
     (I.PERIODIC, I.PERIODIC, I.SPECULAR, I.EXTRAP), dict(nu=0.3)),
    # three v1 columns per lane: mirrored x upwind at the specular side, a zero row behind the
    # diffuse side, specular images of the bottom row
    ("walls_24", dict(nx=9, ny=8, nv1=24, nv2=24),
     (I.DIFFUSE, I.SPECULAR, I.SPECULAR, I.EXTRAP), dict(wall_T=(1.2, 1.0, 1.0, 1.0))),
    # 32^2 (the per-warp flat kernel): zero row behind a diffuse x side, G* exported for the
    # wall kernel at the diffuse top wall
    ("walls_32", dict(nx=7, ny=9, nv1=32, nv2=32),
     (I.SPECULAR, I.DIFFUSE, I.EXTRAP, I.DIFFUSE), dict(wall_T=(1.0, 0.9, 1.0, 1.15))),
    # grids smaller than a CTA's four columns: idle warps in the barriers, halo slots past the
    # edge; one row (periodic y: the cell is its own y neighbour), one column
    ("tiny_16", dict(nx=3, ny=2, nv1=16, nv2=16), (I.PERIODIC, I.PERIODIC, I.SPECULAR, I.SPECULAR), {}),
    ("row_24", dict(nx=5, ny=1, nv1=24, nv2=24), (I.EXTRAP, I.SPECULAR, I.PERIODIC, I.PERIODIC), {}),
    ("column_32", dict(nx=1, ny=6, nv1=32, nv2=32), (I.PERIODIC, I.PERIODIC, I.DIFFUSE, I.EXTRAP),
     dict(wall_T=(1.0, 1.0, 1.1, 1.0))),
    # tall enough for several row segments: with diffuse walls on the bottom and top only, the
    # segments that export the wall rows' G* run first and the wall kernel runs beside the rest
    ("walls_y_segments_24", dict(nx=8, ny=64, nv1=24, nv2=24),
     (I.PERIODIC, I.PERIODIC, I.DIFFUSE, I.DIFFUSE), dict(wall_T=(1.0, 1.0, 1.1, 0.9))),
    ("walls_y_segments_16", dict(nx=12, ny=50, nv1=16, nv2=16),
     (I.EXTRAP, I.SPECULAR, I.DIFFUSE, I.DIFFUSE), dict(wall_T=(1.0, 1.0, 1.2, 1.0))),
    # several row segments with periodic y (the first and last segments' halo rows wrap, and so
    # do the rows whose coefficients are fetched ahead) and with specular y walls (mirrored rows
    # in the first and last segments)
    ("periodic_segments_24", dict(nx=6, ny=64, nv1=24, nv2=24), (I.PERIODIC,) * 4, {}),
    ("specular_segments_16", dict(nx=5, ny=48, nv1=16, nv2=16), (I.SPECULAR,) * 4, {}),
    # moving diffuse walls at the left and bottom (a corner cell with two wall ghosts), the
    # literal wall form of Ghat (no (G - M)/eps term)
    ("walls_literal_24", dict(nx=10, ny=8, nv1=24, nv2=24),
     (I.DIFFUSE, I.EXTRAP, I.DIFFUSE, I.SPECULAR),
     dict(wall_T=(1.1, 1.0, 0.9, 1.0), wall_U=(0.1, 0.0, -0.2, 0.0), wall_keep_es_term=0)),
    # v2 mesh not symmetric about zero: the column-mapped kernel of the 24^2 shape
    ("asym_24", dict(nx=8, ny=9, nv1=24, nv2=24, v2min=-7.0, v2max=9.0),
     (I.EXTRAP, I.EXTRAP, I.PERIODIC, I.PERIODIC), {}),
]


@pytest.mark.parametrize("eps", [1e-2, 1.0])
@pytest.mark.parametrize("name,gk,bc,extra", CASES, ids=[c[0] for c in CASES])
def test_fp32g_against_oracle(name, gk, bc, extra, eps):
    grid = I.Grid(**gk)
    p64 = I.Params(bc=bc, **extra)
    p32 = I.Params(bc=bc, precision=I.PREC_G_FP32, **extra)
    Q = I.smooth_state(grid, seed=len(name), umax=0.25, aniso=0.08)
    G = I.seeded_g(grid, seed=3, amp=0.02)
    dt = O.dt_for_cfl(grid, 0.5, 0.0, I.CFL_SUM)[0]
    n = 12
    Qg, Gg, Hg = run(grid, p32, Q, G, dt, eps, n)
    Qo, Go, Ho = O.step(grid, p64, Q, G, dt, eps, n)
    # g carries FP32 rounding of each step's arithmetic (a few tens of ulp per step, relative to
    # the Maxwellian scale, amplified by 1/eps through (G - M)/eps), macro fields see it through
    # eps * sum c^3 g times dt/dx per step.
    mscale = np.max(Qo[0]) / (2 * np.pi * 0.5)
    gtol = n * 64 * U32 * max(np.max(np.abs(Go)), mscale / eps)
    assert np.max(np.abs(Gg - Go)) <= gtol, (np.max(np.abs(Gg - Go)), gtol)
    eq = q_rel_err(Qg, Qo)
    assert np.all(eq <= n * 64 * U32), eq


def test_fp32g_l1_density_error_vs_fp64_four_quadrant():
    """Four-quadrant Riemann data with a diffuse bottom wall (reduced 128^2 x 24^2): the relative
    L1 density error of FP32 g against the FP64 GPU run stays below 1e-3."""
    pr = I.riemann4_diffuse(n=128, nv=24, eps=1e-2, seed=0, nsteps=60)
    p64 = I.Params(**{**pr.params.__dict__, "precision": I.PREC_FP64})
    p32 = I.Params(**{**pr.params.__dict__, "precision": I.PREC_G_FP32})
    Q64, _, _ = run(pr.grid, p64, pr.Q, pr.G, pr.dt, pr.eps, pr.nsteps)
    Q32, _, _ = run(pr.grid, p32, pr.Q, pr.G, pr.dt, pr.eps, pr.nsteps)
    l1 = np.sum(np.abs(Q32[0] - Q64[0])) / np.sum(np.abs(Q64[0]))
    print("relative L1 density error FP32-g vs FP64:", l1)
    assert l1 <= 1e-3
    assert l1 <= 1e-5  # what the arithmetic actually gives (FP32 round-off, not truncation)


def test_fp32g_full_size_four_quadrant_vs_fp64():
    """The FP32-g benchmark problem at its full size (1024^2 x 24^2, diffuse bottom wall, from
    g = 0 as the benchmark starts it) in the kernel variant the benchmark times: after 20 steps
    the relative L1 density error against the FP64 path stays at the FP32 round-off level, and
    both runs conserve what the diffuse wall and the open sides let them (finite, positive
    density everywhere)."""
    pr = I.riemann4_diffuse(n=1024, nv=24, eps=1e-2, seed=0, nsteps=20)
    p64 = I.Params(**{**pr.params.__dict__, "precision": I.PREC_FP64})
    p32 = I.Params(**{**pr.params.__dict__, "precision": I.PREC_G_FP32})

    def moments(params):  # without copying the 4.8 GB of g back
        with api.Solver(pr.grid, params) as s:
            s.set_state(pr.Q, None)
            s.step(pr.dt, pr.eps, pr.nsteps)
            return s.get_moments(with_H=False)[0]

    Q64, Q32 = moments(p64), moments(p32)
    assert np.all(np.isfinite(Q32)) and np.all(Q32[0] > 0.0)
    l1 = np.sum(np.abs(Q32[0] - Q64[0])) / np.sum(np.abs(Q64[0]))
    print("full size: relative L1 density error FP32-g vs FP64:", l1)
    assert l1 <= 1e-7


def test_fp32g_beyond_32bit_phase_offsets_vs_fp64():
    """The four-quadrant problem at 2048^2 x 24^2 (2.4e9 phase cells: offsets beyond 2^31 in the
    staged FP32-g kernel, its wall export and the FP64 path) after 10 steps: every density finite
    and positive and the relative L1 density error against the FP64 path at round-off level."""
    pr = I.riemann4_diffuse(n=2048, nv=24, eps=1e-2, seed=0, nsteps=10)
    assert pr.grid.nphase > 2 ** 31
    p64 = I.Params(**{**pr.params.__dict__, "precision": I.PREC_FP64})
    p32 = I.Params(**{**pr.params.__dict__, "precision": I.PREC_G_FP32})

    def moments(params):
        with api.Solver(pr.grid, params) as s:
            s.set_state(pr.Q, None)
            s.step(pr.dt, pr.eps, pr.nsteps)
            return s.get_moments(with_H=False)[0]

    Q64, Q32 = moments(p64), moments(p32)
    assert np.all(np.isfinite(Q64)) and np.all(np.isfinite(Q32)) and np.all(Q32[0] > 0.0)
    l1 = np.sum(np.abs(Q32[0] - Q64[0])) / np.sum(np.abs(Q64[0]))
    print("2048^2 x 24^2: relative L1 density error FP32-g vs FP64:", l1)
    assert l1 <= 1e-7


@pytest.mark.parametrize("bc", [(I.EXTRAP, I.EXTRAP, I.DIFFUSE, I.EXTRAP),
                                (I.DIFFUSE, I.SPECULAR, I.SPECULAR, I.DIFFUSE)])
def test_pipelined_steps_equal_single_steps(bc):
    """Several FP32-g steps in one call (macro x1 of each step on a side stream beside the
    phase-space kernel) equal one call per step bit for bit, with diffuse walls on the bottom,
    top and x sides."""
    g = I.Grid(nx=96, ny=256, nv1=24, nv2=24)
    p = I.Params(nu=-0.5, bc=bc, wall_T=(1.1, 1.0, 0.9, 1.2), wall_U=(0.1, 0.0, 0.2, -0.1),
                 precision=I.PREC_G_FP32)
    Q = I.smooth_state(g, seed=5, umax=0.2, aniso=0.05)
    dt = api.mm_dt_for_cfl(g, 0.5, 0.0, I.CFL_SUM)[0]
    out = []
    for calls in ((10,), (1,) * 10):
        with api.Solver(g, p) as s:
            s.set_state(Q, None)
            for n in calls:
                s.step(dt, 1e-2, n)
            Qa, Ha = s.get_moments()
            Ga = s.get_g()
        out.append((Qa, Ha, Ga))
    (Qa, Ha, Ga), (Qb, Hb, Gb) = out
    assert np.array_equal(Qa, Qb) and np.array_equal(Ha, Hb) and np.array_equal(Ga, Gb)
