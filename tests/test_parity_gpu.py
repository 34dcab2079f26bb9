"""GPU parity: the CUDA path (through the C ABI) against the plain FP64 CPU oracle.

Macro fields must agree to 1e-12 in the per-component metric of helpers.q_rel_err; g and the
heat flux are compared too.  Cases span several CTAs and ragged sizes (odd cell counts, velocity
meshes whose v1 size does not fill whole warps), every boundary kind, anisotropic pressure
tensors and non-zero initial g, the full 1D-2V shock-tube run, and the full 256^2 x 32^2
specular workload through sampled one-step windows.
"""
import zlib

import numpy as np
import pytest

from helpers import q_rel_err
from oracle import oracle as O
from paper_2509_21832_gb300 import api
from paper_2509_21832_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_Q = 1e-12
ULP = 2.220446049250313e-16


def g_floor(Q, eps):
    """Absolute rounding floor of g: g carries (G - M)/eps, so a few-ulp difference in the two
    Gaussians (evaluated in different but equivalent forms on each side) is amplified by 1/eps."""
    rho = Q[0]
    T = (Q[3] + Q[5] - (Q[1] ** 2 + Q[2] ** 2) / rho) / (2 * rho)
    return 64 * ULP * np.max(rho / (2 * np.pi * T)) / eps


def h_floor(Q):
    """Absolute rounding floor of H = eps dv^2 sum c^3 g: the same few-ulp Gaussian differences,
    times eps/eps, weighted by |c|^3 (E|c|^3 = 3.76 T^1.5 for the 2D Maxwellian)."""
    rho = Q[0]
    T = (Q[3] + Q[5] - (Q[1] ** 2 + Q[2] ** 2) / rho) / (2 * rho)
    return 64 * ULP * 4.0 * np.max(rho * T ** 1.5)


def run_gpu(grid, params, Q, G, dt, eps, nsteps):
    with api.Solver(grid, params) as s:
        s.set_state(Q, G)
        s.step(dt, eps, nsteps)
        s.sync()
        Qg, Hg = s.get_moments()
        Gg = s.get_g()
    return Qg, Gg, Hg


def check(grid, params, Q, G, dt, eps, nsteps, tol_q=TOL_Q, tol_g=1e-11):
    Qg, Gg, Hg = run_gpu(grid, params, Q, G, dt, eps, nsteps)
    Qo, Go, Ho = O.step(grid, params, Q, G, dt, eps, nsteps)
    eq = q_rel_err(Qg, Qo)
    assert np.all(eq <= tol_q), eq
    gtol = max(tol_g * np.max(np.abs(Go)), g_floor(Qo, eps))
    assert np.max(np.abs(Gg - Go)) <= gtol, (np.max(np.abs(Gg - Go)), gtol)
    htol = max(tol_g * np.max(np.abs(Ho)), h_floor(Qo))
    assert np.max(np.abs(Hg - Ho)) <= htol, (np.max(np.abs(Hg - Ho)), htol)
    return eq


def test_sod_1d2v_full_run():
    pr = I.sod_1d2v()
    eq = check(pr.grid, pr.params, pr.Q, pr.G, pr.dt, pr.eps, pr.nsteps)
    print("sod 1d2v: max rel err", eq.max())


CASES = [
    # name, grid kwargs, bc, extra params
    ("periodic_24", dict(nx=13, ny=11, nv1=24, nv2=24), (I.PERIODIC,) * 4, {}),
    ("extrap_16", dict(nx=9, ny=14, nv1=16, nv2=16), (I.EXTRAP,) * 4, {}),
    ("specular_32", dict(nx=10, ny=7, nv1=32, nv2=32), (I.SPECULAR,) * 4, {}),
    ("mixed_diffuse_24", dict(nx=12, ny=9, nv1=24, nv2=24),
     (I.EXTRAP, I.EXTRAP, I.DIFFUSE, I.EXTRAP), dict(wall_T=(1.0, 1.0, 1.1, 1.0))),
    ("cavity_20", dict(nx=8, ny=8, nv1=20, nv2=20, v1min=-5, v1max=5, v2min=-5, v2max=5),
     (I.DIFFUSE,) * 4, dict(wall_T=(1.0,) * 4, wall_U=(0.0, 0.0, 0.0, 0.16), nu=-1.0,
                             tau_model=I.TAU_HARDSPHERE2D)),
    ("cavity_literal_14", dict(nx=7, ny=6, nv1=14, nv2=14, v1min=-5, v1max=5, v2min=-5, v2max=5),
     (I.DIFFUSE,) * 4, dict(wall_T=(0.9, 1.1, 1.0, 1.0), wall_U=(0.05, -0.1, 0.0, 0.2),
                             wall_keep_es_term=0)),
    ("odd_mesh_17x15", dict(nx=6, ny=5, nv1=17, nv2=15, v1min=-6, v1max=6, v2min=-6, v2max=6),
     (I.PERIODIC, I.PERIODIC, I.SPECULAR, I.DIFFUSE), dict(tau_model=I.TAU_PRESSURE, nu=0.3)),
    ("asym_mesh_extrap", dict(nx=5, ny=6, nv1=12, nv2=22, v1min=-5, v1max=7, v2min=-7, v2max=6),
     (I.EXTRAP,) * 4, dict(tau_model=I.TAU_CONST, tau0=0.8)),
]


@pytest.mark.parametrize("eps", [1e-3, 1e-1, 5.0])
@pytest.mark.parametrize("name,gk,bc,extra", CASES, ids=[c[0] for c in CASES])
def test_small_cases(name, gk, bc, extra, eps):
    grid = I.Grid(**gk)
    params = I.Params(bc=bc, **extra)
    Q = I.smooth_state(grid, seed=zlib.crc32(name.encode()) % 1000, umax=0.25, aniso=0.08)
    G = I.seeded_g(grid, seed=7, amp=0.02)
    dt = O.dt_for_cfl(grid, 0.5, 0.0, I.CFL_SUM)[0]
    check(grid, params, Q, G, dt, eps, 12)


def test_one_cell_and_one_row():
    g = I.Grid(nx=1, ny=1, nv1=8, nv2=8)
    p = I.Params(bc=(I.PERIODIC,) * 4)
    Q = I.q_from_prims(np.full((1, 1), 1.1), 0.2, -0.1, 0.9, 0.05, 0.02)
    check(g, p, Q, I.seeded_g(g, 3), 1e-3, 0.05, 5)
    g = I.Grid(nx=9, ny=1, nv1=8, nv2=8)
    p = I.Params(bc=(I.SPECULAR, I.DIFFUSE, I.PERIODIC, I.PERIODIC))
    Q = I.smooth_state(g, seed=5)
    check(g, p, Q, I.seeded_g(g, 4), 5e-3, 0.05, 5)


def test_long_velocity_mesh_large_shared_tables():
    """nv2 = 600: the y kernel's shared tables exceed 48 KB."""
    g = I.Grid(nx=3, ny=4, nv1=2, nv2=600, v1min=-6, v1max=6, v2min=-10, v2max=10)
    p = I.Params(bc=(I.PERIODIC,) * 4)
    Q = I.smooth_state(g, seed=9, umax=0.2)
    dt = O.dt_for_cfl(g, 0.5, 0.0, I.CFL_SUM)[0]
    check(g, p, Q, I.seeded_g(g, 8), dt, 0.1, 3)


def test_zero_steps_is_identity():
    g = I.Grid(nx=5, ny=4, nv1=8, nv2=8)
    p = I.Params(bc=(I.PERIODIC,) * 4)
    Q = I.smooth_state(g, seed=1)
    G = I.seeded_g(g, 2)
    Qg, Gg, _ = run_gpu(g, p, Q, G, 1e-3, 0.1, 0)
    assert np.array_equal(Qg, Q) and np.array_equal(Gg, G)


def test_checkpoint_resume_bitwise():
    g = I.Grid(nx=11, ny=9, nv1=16, nv2=16)
    p = I.Params(bc=(I.SPECULAR, I.SPECULAR, I.EXTRAP, I.DIFFUSE))
    Q = I.smooth_state(g, seed=17)
    G = I.seeded_g(g, 18)
    dt = O.dt_for_cfl(g, 0.5, 0.0, I.CFL_SUM)[0]
    Qa, Ga, Ha = run_gpu(g, p, Q, G, dt, 0.02, 10)
    Q5, G5, _ = run_gpu(g, p, Q, G, dt, 0.02, 5)
    Qb, Gb, Hb = run_gpu(g, p, Q5, G5, dt, 0.02, 5)
    assert np.array_equal(Qa, Qb) and np.array_equal(Ga, Gb) and np.array_equal(Ha, Hb)


@pytest.mark.parametrize("prec", [I.PREC_FP64, I.PREC_G_FP32])
def test_nonphysical_state_is_reported(prec):
    """A negative density is reported as MM_ERR_NONPHYSICAL by either precision's fields
    kernel."""
    g = I.Grid(nx=6, ny=5, nv1=8, nv2=8)
    p = I.Params(bc=(I.PERIODIC,) * 4, precision=prec)
    Q = I.smooth_state(g, seed=1)
    Q[0, 2, 3] = -1.0
    with api.Solver(g, p) as s:
        s.set_state(Q)
        s.step(1e-3, 0.1, 1)
        with pytest.raises(api.MMError) as e:
            s.sync()
        assert e.value.status == api.MM_ERR_NONPHYSICAL


def test_step_before_state_and_bad_dt():
    g = I.Grid(nx=4, ny=4, nv1=8, nv2=8)
    with api.Solver(g, I.Params()) as s:
        with pytest.raises(api.MMError) as e:
            s.step(1e-3, 0.1, 1)
        assert e.value.status == api.MM_ERR_STATE
        s.set_state(I.smooth_state(g, 1))
        for dt, eps in ((0.0, 0.1), (1e-3, -1.0), (float("nan"), 0.1)):
            with pytest.raises(api.MMError) as e:
                s.step(dt, eps, 1)
            assert e.value.status == api.MM_ERR_INVALID_ARG


def test_conservation_periodic_gpu():
    g = I.Grid(nx=64, ny=48, nv1=24, nv2=24)
    p = I.Params(bc=(I.PERIODIC,) * 4)
    Q = I.smooth_state(g, seed=3)
    dt = O.dt_for_cfl(g, 0.5, 0.0, I.CFL_SUM)[0]
    Qg, _, _ = run_gpu(g, p, Q, I.seeded_g(g, 4), dt, 0.01, 50)
    for m in (0, 1, 2):
        assert abs(Qg[m].sum() - Q[m].sum()) <= 1e-13 * Q[0].sum() * 1
    assert abs((Qg[3] + Qg[5]).sum() - (Q[3] + Q[5]).sum()) <= 1e-13 * (Q[3] + Q[5]).sum()


# ---------------------------------------------------------------------------------------------
# full-size 256^2 x 32^2 specular workload: sampled one-step windows against the oracle
# ---------------------------------------------------------------------------------------------
def _window(pr, Q, G, i0, j0, w):
    g = pr.grid
    dx, dy = (g.x1 - g.x0) / g.nx, (g.y1 - g.y0) / g.ny
    i0c, j0c = max(0, i0), max(0, j0)
    i1c, j1c = min(g.nx, i0 + w), min(g.ny, j0 + w)
    sub = I.Grid(nx=i1c - i0c, ny=j1c - j0c, x0=g.x0 + i0c * dx, x1=g.x0 + i1c * dx,
                 y0=g.y0 + j0c * dy, y1=g.y0 + j1c * dy, nv1=g.nv1, nv2=g.nv2, v1min=g.v1min,
                 v1max=g.v1max, v2min=g.v2min, v2max=g.v2max)
    bc = list(pr.params.bc)
    if i0c > 0:
        bc[0] = I.EXTRAP
    if i1c < g.nx:
        bc[1] = I.EXTRAP
    if j0c > 0:
        bc[2] = I.EXTRAP
    if j1c < g.ny:
        bc[3] = I.EXTRAP
    p = I.Params(**{**pr.params.__dict__, "bc": tuple(bc)})
    return sub, p, np.ascontiguousarray(Q[:, j0c:j1c, i0c:i1c]), \
        np.ascontiguousarray(G[j0c:j1c, i0c:i1c]), (i0c, j0c)


@pytest.mark.parametrize("eps", [1e-3, 1e-1])
def test_full_size_bump_specular_sampled(eps):
    pr = I.bump_specular(eps=eps, seed=0)
    with api.Solver(pr.grid, pr.params) as s:
        s.set_state(pr.Q, pr.G)
        s.step(pr.dt, pr.eps, 8)
        Q8, _ = s.get_moments()
        G8 = s.get_g()
        s.step(pr.dt, pr.eps, 1)
        Q9, H9 = s.get_moments()
        G9 = s.get_g()
    x0, y0 = pr.meta["x0"]
    ic, jc = int(x0 * pr.grid.nx), int(y0 * pr.grid.ny)
    targets = [(0, 0), (255, 0), (0, 255), (255, 255), (128, 0), (0, 77), (ic, jc),
               (ic + 9, jc - 5), (200, 31)]
    w = 7
    gtol = max(1e-11 * np.max(np.abs(G9)), g_floor(Q9, pr.eps))
    htol = max(1e-11 * np.max(np.abs(H9)), h_floor(Q9))
    for (ti, tj) in targets:
        sub, p, Qw, Gw, (oi, oj) = _window(pr, Q8, G8, ti - w // 2, tj - w // 2, w)
        Qo, Go, Ho = O.step(sub, p, Qw, Gw, pr.dt, pr.eps, 1)
        li, lj = ti - oi, tj - oj
        qg, qo = Q9[:, tj, ti], Qo[:, lj, li]
        scale = max(np.max(np.abs(Qo[0])), 1.0)
        assert np.max(np.abs(qg - qo)) <= TOL_Q * scale, (ti, tj, qg - qo)
        # g and H errors relative to the field's global scale (far from the bump g is round-off)
        assert np.max(np.abs(G9[tj, ti] - Go[lj, li])) <= gtol, (ti, tj)
        assert np.max(np.abs(H9[:, tj, ti] - Ho[:, lj, li])) <= htol, (ti, tj)
    # properties that hold at any size: specular walls conserve mass and energy to round-off
    assert abs(Q9[0].sum() - pr.Q[0].sum()) <= 1e-13 * pr.Q[0].sum()
    assert abs((Q9[3] + Q9[5]).sum() - (pr.Q[3] + pr.Q[5]).sum()) <= 1e-13 * (pr.Q[3] + pr.Q[5]).sum()


def test_beyond_32bit_phase_offsets_sampled():
    """More than 2^31 phase cells (the bump at 1536^2 x 32^2: 2.4e9 phase cells, about 40 GB on
    the device, in the benchmark's launch configuration): one-step windows against the oracle,
    among them cells in the top rows whose phase-space offsets exceed 2^31, plus mass and energy
    conservation.  The state lives in CUDA tensors (mm_create_borrowed), so only the windows
    cross to the host."""
    import torch
    pr = I.bump_specular(n=1536, nv=32, eps=1e-1, seed=0)
    g = pr.grid
    nc, nv = g.nx * g.ny, g.nv1 * g.nv2
    assert nc * nv > 2 ** 31
    Qt = torch.empty(6 * nc, dtype=torch.float64, device="cuda")
    Gt = torch.empty(nc * nv, dtype=torch.float64, device="cuda")
    St = torch.empty(api.mm_scratch_bytes(g, pr.params), dtype=torch.uint8, device="cuda")
    Gv = Gt.view(g.ny, g.nx, g.nv2, g.nv1)
    x0, y0 = pr.meta["x0"]
    ic, jc = int(x0 * g.nx), int(y0 * g.ny)
    targets = [(0, 0), (g.nx - 1, g.ny - 1), (g.nx - 1, 0), (0, g.ny - 1), (ic, jc),
               (700, 1500), (1200, 1420), (g.nx // 2, g.ny - 1)]
    w = 7
    with api.Solver(g, pr.params, borrow=(Qt, Gt, St)) as s:
        s.set_state(pr.Q, None)
        s.step(pr.dt, pr.eps, 8)
        s.sync()
        Q8 = Qt.view(6, g.ny, g.nx).cpu().numpy()
        wins = {}
        for (ti, tj) in targets:
            i0, j0 = max(0, ti - w // 2), max(0, tj - w // 2)
            i1, j1 = min(g.nx, ti - w // 2 + w), min(g.ny, tj - w // 2 + w)
            wins[(ti, tj)] = (i0, j0, i1, j1, Gv[j0:j1, i0:i1].cpu().numpy())
        s.step(pr.dt, pr.eps, 1)
        Q9, H9 = s.get_moments()
        torch.cuda.synchronize()
        gmax = max(float(Gt[k:k + (1 << 27)].abs().max()) for k in range(0, nc * nv, 1 << 27))
        G9w = {t: Gv[t[1], t[0]].cpu().numpy() for t in targets}
    gtol = max(1e-11 * gmax, g_floor(Q9, pr.eps))
    htol = max(1e-11 * np.max(np.abs(H9)), h_floor(Q9))
    dx, dy = (g.x1 - g.x0) / g.nx, (g.y1 - g.y0) / g.ny
    for (ti, tj), (i0, j0, i1, j1, Gw) in wins.items():
        sub = I.Grid(nx=i1 - i0, ny=j1 - j0, x0=g.x0 + i0 * dx, x1=g.x0 + i1 * dx,
                     y0=g.y0 + j0 * dy, y1=g.y0 + j1 * dy, nv1=g.nv1, nv2=g.nv2,
                     v1min=g.v1min, v1max=g.v1max, v2min=g.v2min, v2max=g.v2max)
        bc = list(pr.params.bc)
        bc[0] = bc[0] if i0 == 0 else I.EXTRAP
        bc[1] = bc[1] if i1 == g.nx else I.EXTRAP
        bc[2] = bc[2] if j0 == 0 else I.EXTRAP
        bc[3] = bc[3] if j1 == g.ny else I.EXTRAP
        p = I.Params(**{**pr.params.__dict__, "bc": tuple(bc)})
        Qo, Go, Ho = O.step(sub, p, np.ascontiguousarray(Q8[:, j0:j1, i0:i1]), Gw, pr.dt,
                            pr.eps, 1)
        li, lj = ti - i0, tj - j0
        scale = max(np.max(np.abs(Qo[0])), 1.0)
        assert np.max(np.abs(Q9[:, tj, ti] - Qo[:, lj, li])) <= TOL_Q * scale, (ti, tj)
        assert np.max(np.abs(G9w[(ti, tj)] - Go[lj, li])) <= gtol, (ti, tj)
        assert np.max(np.abs(H9[:, tj, ti] - Ho[:, lj, li])) <= htol, (ti, tj)
    assert abs(Q9[0].sum() - pr.Q[0].sum()) <= 1e-13 * pr.Q[0].sum()
    assert abs((Q9[3] + Q9[5]).sum() - (pr.Q[3] + pr.Q[5]).sum()) <= 1e-13 * (pr.Q[3] + pr.Q[5]).sum()


@pytest.mark.parametrize("bc,u,nv,prec", [
    ((I.PERIODIC,) * 4, (0.4, -0.3), 32, I.PREC_FP64),
    ((I.SPECULAR,) * 4, (0.0, 0.0), 32, I.PREC_FP64),
    ((I.EXTRAP,) * 4, (0.3, 0.2), 24, I.PREC_FP64),
    ((I.DIFFUSE,) * 4, (0.0, 0.0), 16, I.PREC_FP64),
    ((I.SPECULAR, I.SPECULAR, I.PERIODIC, I.PERIODIC), (0.0, 0.1), 24, I.PREC_G_FP32),
    ((I.DIFFUSE,) * 4, (0.0, 0.0), 24, I.PREC_G_FP32),
])
def test_global_maxwellian_is_preserved_gpu(bc, u, nv, prec):
    """A global Maxwellian (uniform rho, u, T; g = 0; walls at rest at the gas temperature) is a
    fixed point of the scheme: on the GPU, Q stays put to round-off and g stays at round-off, for
    every boundary kind that admits it, in both precisions of g (Sections 5.3-5.4: Z = 0 and
    Zhat = 0 for an exact Maxwellian, Ghat = 0 without gradients, the KFVS faces cancel)."""
    g = I.Grid(nx=14, ny=11, nv1=nv, nv2=nv)
    p = I.Params(nu=-0.5, bc=bc, wall_T=(0.8,) * 4, precision=prec)
    Q0 = I.q_from_prims(np.full((11, 14), 1.3), u[0], u[1], 0.8)
    dt = O.dt_for_cfl(g, 0.5, 0.0, I.CFL_SUM)[0]
    with api.Solver(g, p) as s:
        s.set_state(Q0, None)
        s.step(dt, 1e-2, 25)
        Q, _ = s.get_moments()
        G = s.get_g()
    tol_q = 1e-13 if prec == I.PREC_FP64 else 1e-6
    assert np.max(np.abs(Q - Q0)) < tol_q, np.max(np.abs(Q - Q0))
    # g of an exact equilibrium is round-off: FP64 sums, or FP32 storage of round-off
    assert np.max(np.abs(G)) < (1e-11 if prec == I.PREC_FP64 else 1e-5), np.max(np.abs(G))


@pytest.mark.parametrize("eps", [1e-8, 1e30])
@pytest.mark.parametrize("name,gk,bc,extra", [CASES[0], CASES[2], CASES[3]],
                         ids=[CASES[0][0], CASES[2][0], CASES[3][0]])
def test_extreme_knudsen_numbers(name, gk, bc, extra, eps):
    """The asymptotic-preserving end (eps = 1e-8: g^{n+1} is Ghat^n up to O(eps), the relaxation
    weights are 0 and 1 to within 1e-8) and free streaming (eps = 1e30: the collision weights are
    exactly 1 and 0 in FP64, as in the paper's collisionless check, which starts from g = 0:
    f = M + eps g, so a g of order one would be a non-physical f there) against the oracle."""
    grid = I.Grid(**gk)
    params = I.Params(bc=bc, **extra)
    Q = I.smooth_state(grid, seed=zlib.crc32(name.encode()) % 1000, umax=0.25, aniso=0.08)
    G = I.seeded_g(grid, seed=7, amp=0.02) if eps < 1.0 else I.zero_g(grid)
    dt = O.dt_for_cfl(grid, 0.5, 0.0, I.CFL_SUM)[0]
    check(grid, params, Q, G, dt, eps, 12)


@pytest.mark.parametrize("nv1,nv2,bc", [
    (512, 4, (I.SPECULAR,) * 4),      # the widest v1 mesh: 512-thread CTAs, 16-warp reductions
    (1, 1024, (I.PERIODIC,) * 4),     # one v1 column, the longest v2 mesh: 107 KB of y tables
    (1, 1024, (I.SPECULAR, I.SPECULAR, I.DIFFUSE, I.EXTRAP)),
])
def test_velocity_mesh_limits(nv1, nv2, bc):
    """The ends of the accepted velocity meshes (nv1 in 1..512, nv2 in 1..1024) against the
    oracle on a 3 x 2 grid."""
    grid = I.Grid(nx=3, ny=2, nv1=nv1, nv2=nv2)
    params = I.Params(bc=bc, wall_T=(1.0, 1.0, 1.05, 1.0))
    Q = I.smooth_state(grid, seed=nv1 + nv2, umax=0.2, aniso=0.05)
    G = I.seeded_g(grid, seed=3, amp=0.02)
    dt = O.dt_for_cfl(grid, 0.5, 0.0, I.CFL_SUM)[0]
    check(grid, params, Q, G, dt, 1e-2, 4)
