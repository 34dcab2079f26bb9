"""Pins of the plain FP64 CPU oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: numbers printed in the paper,
closed forms, brute-force quadrature, an independently coded TR-BDF2 step, the exact Euler
Riemann solution, or invariants (conservation, preserved equilibria).  A plausible slip in the
oracle (a dropped term, a flipped sign, a swapped index, the downwind KFVS reading) fails at
least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_21832_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------------------------------------
# time-step rule: step counts printed in Sections 4.2 and 6.2
# ---------------------------------------------------------------------------------------------
def test_dt_rule_matches_printed_step_counts():
    with open(os.path.join(GOLDEN, "dt_rule.json")) as f:
        fx = json.load(f)
    for c in fx["cases"]:
        g = I.Grid(nx=c["nx"], ny=c["ny"], x0=c["x0"], x1=c["x1"], y0=c["y0"], y1=c["y1"],
                   nv1=14, nv2=14, v1min=-c["vmax"], v1max=c["vmax"], v2min=-c["vmax"],
                   v2max=c["vmax"])
        dt, n = O.dt_for_cfl(g, c["cfl"], c["t_final"], c["form"])
        assert n == c["nsteps"], c["name"]
        assert abs(dt - c["dt"]) <= c["dt_rtol"] * c["dt"], c["name"]
        dx = (c["x1"] - c["x0"]) / c["nx"]
        dy = (c["y1"] - c["y0"]) / c["ny"]
        cfl = dt * c["vmax"] / dx if c["ny"] == 1 else dt * (c["vmax"] / dx + c["vmax"] / dy)
        assert abs(cfl - c["cfl_after"]) <= c["cfl_rtol"] * c["cfl_after"], c["name"]
    # the min form of Eq. (CFL-2D-part1) gives 107 steps for the cylindrical problem
    c = fx["cases"][1]
    g = I.Grid(nx=320, ny=320, x0=-1, x1=1, y0=-1, y1=1, v1min=-9, v1max=9, v2min=-9, v2max=9)
    assert O.dt_for_cfl(g, 0.95, 0.07, I.CFL_MIN)[1] == 107
    # the 1D-2V Sod workload: dt = 0.5 * (1/200) / 8 and exactly 640 steps to t = 0.2
    p = I.sod_1d2v()
    dt, n = O.dt_for_cfl(p.grid, 0.5, 0.2, I.CFL_SUM)
    assert n == 640 and abs(dt - 3.125e-4) < 1e-18


# ---------------------------------------------------------------------------------------------
# KFVS half-range fluxes against brute-force quadrature of int v_d m(v) G dv over a half space
# ---------------------------------------------------------------------------------------------
def _gauss_legendre_box(lo, hi, n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (hi - lo) * x + 0.5 * (hi + lo), 0.5 * (hi - lo) * w


def _half_flux_quadrature(q, direction, positive):
    rho = q[0]
    u = np.array([q[1], q[2]]) / rho
    P = np.array([[q[3] - rho * u[0] ** 2, q[4] - rho * u[0] * u[1]],
                  [q[4] - rho * u[0] * u[1], q[5] - rho * u[1] ** 2]])
    Th = P / rho
    Ti = np.linalg.inv(Th)
    L = 14.0 * math.sqrt(max(Th[0, 0], Th[1, 1]))
    d = direction - 1
    o = 1 - d
    # normal velocity on (0, u_d + L) or (u_d - L, 0); tangential on u_o -+ L, split at u_o
    if positive:
        vn, wn = _gauss_legendre_box(0.0, max(u[d] + L, 1e-3), 160)
    else:
        vn, wn = _gauss_legendre_box(min(u[d] - L, -1e-3), 0.0, 160)
    vt1, wt1 = _gauss_legendre_box(u[o] - L, u[o], 120)
    vt2, wt2 = _gauss_legendre_box(u[o], u[o] + L, 120)
    vt, wt = np.concatenate([vt1, vt2]), np.concatenate([wt1, wt2])
    VN, VT = np.meshgrid(vn, vt, indexing="ij")
    W = wn[:, None] * wt[None, :]
    v = [None, None]
    v[d], v[o] = VN, VT
    c1, c2 = v[0] - u[0], v[1] - u[1]
    quad = Ti[0, 0] * c1 * c1 + 2 * Ti[0, 1] * c1 * c2 + Ti[1, 1] * c2 * c2
    G = rho / (2 * math.pi * math.sqrt(np.linalg.det(Th))) * np.exp(-0.5 * quad)
    m = [np.ones_like(c1), v[0], v[1], v[0] ** 2, v[0] * v[1], v[1] ** 2]
    return np.array([np.sum(W * v[d] * mm * G) for mm in m])


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_kfvs_half_fluxes_match_quadrature(seed):
    rng = I.SplitMix64(seed)
    rho = rng.uniform(0.3, 2.0)
    u1, u2 = rng.uniform(-1.5, 1.5), rng.uniform(-1.5, 1.5)
    T = rng.uniform(0.4, 1.6)
    a, s = rng.uniform(-0.3, 0.3) * T, rng.uniform(-0.3, 0.3) * T
    q = I.q_from_prims(np.array(rho), u1, u2, T, a, s)
    for direction in (1, 2):
        Fp, Fm = O.kfvs_half(q, direction)
        Rp = _half_flux_quadrature(q, direction, True)
        Rm = _half_flux_quadrature(q, direction, False)
        scale = np.abs(Rp) + np.abs(Rm) + 1e-300
        assert np.all(np.abs(Fp - Rp) <= 1e-11 * scale.max()), (direction, Fp, Rp)
        assert np.all(np.abs(Fm - Rm) <= 1e-11 * scale.max()), (direction, Fm, Rm)


# ---------------------------------------------------------------------------------------------
# projector Pi_M: reproduces the null-space basis and annihilates a function orthogonal to it
# ---------------------------------------------------------------------------------------------
def test_projector_identities():
    g = I.Grid(nx=1, ny=1, nv1=32, nv2=32)
    rho, u1, u2, T = 1.3, 0.4, -0.25, 0.9
    v1, v2 = g.v1()[None, :], g.v2()[:, None]
    c1, c2 = v1 - u1, v2 - u2
    M = rho / (2 * math.pi * T) * np.exp(-(c1 ** 2 + c2 ** 2) / (2 * T))
    basis = [np.ones_like(c1 * c2), c1 / math.sqrt(T) + 0 * c2, c2 / math.sqrt(T) + 0 * c1,
             (c1 ** 2 + c2 ** 2) / (2 * T) - 1]
    for b in basis:
        F = b * M
        PF = O.project(g, rho, u1, u2, T, F)
        assert np.max(np.abs(PF - F)) <= 1e-11 * np.max(np.abs(F))
    # a Hermite function of degree 3 in c1 has zero projection
    h3 = (c1 / math.sqrt(T)) ** 3 - 3 * c1 / math.sqrt(T) + 0 * c2
    PF = O.project(g, rho, u1, u2, T, h3 * M)
    assert np.max(np.abs(PF)) <= 1e-11 * np.max(np.abs(h3 * M))
    # idempotence on an arbitrary function
    F = np.cos(v1 * 0.7) * np.exp(-0.3 * v2 ** 2) + 0.1 * v1 * v2 * np.exp(-0.5 * (v1 ** 2 + v2 ** 2))
    P1 = O.project(g, rho, u1, u2, T, F)
    P2 = O.project(g, rho, u1, u2, T, P1)
    assert np.max(np.abs(P2 - P1)) <= 1e-11 * np.max(np.abs(P1))


# ---------------------------------------------------------------------------------------------
# TR-BDF2 factor W against an independently coded two-stage TR-BDF2 step (gamma = 1/2)
# ---------------------------------------------------------------------------------------------
def _trbdf2_scalar(lam, h):
    """y' = -lam y over one step h: trapezoid to h/2, then BDF2 on (0, h/2, h); returns y(h)/y0."""
    y0 = 1.0
    y1 = y0 * (1 - lam * h / 4) / (1 + lam * h / 4)
    return (4 * y1 - y0) / 3 / (1 + lam * h / 3)


@pytest.mark.parametrize("eps", [1e-6, 1e-3, 1e-1, 10.0, 1e30])
def test_trbdf2_factor(eps):
    for tau, nu, dt in [(1.0, -0.5, 1e-3), (0.7, 0.0, 4e-2), (2.0, -1.0, 1e-4)]:
        W = O.trbdf2_W(tau, nu, eps, dt)
        lam = tau * (1 - nu) / eps     # decay rate of P11-P22 and P12 (Eq. 5-40)
        ref = _trbdf2_scalar(lam, dt / 2)
        assert abs(W - ref) <= 1e-14 * max(1.0, abs(ref))
    # L-stability: W -> 0 as eps -> 0; W -> 1 as eps -> infinity
    assert abs(O.trbdf2_W(1.0, -0.5, 1e-12, 1e-2)) < 1e-8
    assert abs(O.trbdf2_W(1.0, -0.5, 1e30, 1e-2) - 1.0) < 1e-15


# ---------------------------------------------------------------------------------------------
# diffuse-wall densities: zero net mass flux through the wall
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [5, 6, 7])
def test_wall_density_zero_mass_flux(seed):
    rng = I.SplitMix64(seed)
    rho = rng.uniform(0.5, 2.0)
    u1, u2 = rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8)
    T = rng.uniform(0.5, 1.5)
    a, s = rng.uniform(-0.2, 0.2) * T, rng.uniform(-0.2, 0.2) * T
    q = I.q_from_prims(np.array(rho), u1, u2, T, a, s)
    Th = np.array([q[3] / rho - u1 * u1, q[5] / rho - u2 * u2])
    Tw = rng.uniform(0.6, 1.4)
    for d, (ua, Taa) in enumerate([(u1, Th[0]), (u2, Th[1])]):
        # wall on the low side: the wall emits v_d > 0, the cell loses its v_d < 0 half
        out_low = _half_flux_quadrature(q, d + 1, False)[0]
        rw = rho * O.wall_R(ua, Taa, Tw, -1)
        assert abs(rw * math.sqrt(Tw / (2 * math.pi)) + out_low) < 1e-12
        # wall on the high side
        out_high = _half_flux_quadrature(q, d + 1, True)[0]
        rw = rho * O.wall_R(ua, Taa, Tw, +1)
        assert abs(-rw * math.sqrt(Tw / (2 * math.pi)) + out_high) < 1e-12


# ---------------------------------------------------------------------------------------------
# ES Gaussian in Ghat: in the space-homogeneous state, eps * (second moments of Ghat) equals
# rho (Tcal - T I) = nu (P - p I)  (Eq. 2-19, Eq. 5-75); its mass and momentum vanish
# ---------------------------------------------------------------------------------------------
def test_ghat_es_term_moments():
    g = I.Grid(nx=3, ny=3, nv1=40, nv2=40, v1min=-10, v1max=10, v2min=-10, v2max=10)
    for nu in (-0.5, -1.0, 0.3):
        p = I.Params(nu=nu, bc=(I.PERIODIC,) * 4)
        rho, u1, u2, T, a, s = 1.2, 0.3, -0.2, 0.9, 0.15, -0.1
        Q = I.q_from_prims(np.full((3, 3), rho), u1, u2, T, a, s)
        eps = 0.37
        Gh = O.ghat(g, p, Q, eps)[1, 1]
        v1, v2 = g.v1()[None, :], g.v2()[:, None]
        c1, c2 = v1 - u1, v2 - u2
        dv = (20.0 / 40) ** 2
        assert abs(np.sum(Gh) * dv) < 1e-12
        assert abs(np.sum(c1 * Gh) * dv) < 1e-12 and abs(np.sum(c2 * Gh) * dv) < 1e-12
        P11, P12, P22 = rho * (T + a), rho * s, rho * (T - a)
        pr = 0.5 * (P11 + P22)
        assert abs(eps * np.sum(c1 * c2 * Gh) * dv - nu * P12) < 1e-12
        assert abs(eps * np.sum((c1 ** 2 - c2 ** 2) * Gh) * dv - nu * (P11 - P22)) < 1e-12
        assert abs(eps * np.sum((c1 ** 2 + c2 ** 2) * Gh) * dv) < 1e-12
        assert abs(pr - rho * T) < 1e-14


# ---------------------------------------------------------------------------------------------
# Ghat transport term converges to -(1/tau)(I - Pi)[v . grad M] computed with exact derivatives
# (Eq. 5-69): pins B, C and the discrete sigma and grad T of Eq. (5-97more)
# ---------------------------------------------------------------------------------------------
def _fields(x, y):
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    u1 = 0.3 * np.cos(2 * np.pi * x + 0.4) * np.sin(2 * np.pi * y)
    u2 = 0.25 * np.sin(2 * np.pi * (x + y))
    T = 1.0 + 0.15 * np.cos(2 * np.pi * x) + 0.1 * np.sin(2 * np.pi * y + 1.0)
    return rho, u1, u2, T


def test_ghat_transport_term_converges_to_analytic_projection():
    p = I.Params(nu=-0.5, bc=(I.PERIODIC,) * 4, tau_model=I.TAU_CONST, tau0=1.0)
    errs = []
    for n in (16, 32, 64):
        # dy = (2/3) dx, so that a dx taken for dy in the discrete gradients shows
        g = I.Grid(nx=n, ny=3 * n // 2, nv1=32, nv2=32)
        x, y = np.meshgrid(g.xc(), g.yc())
        rho, u1, u2, T = _fields(x, y)
        Q = I.q_from_prims(rho, u1, u2, T)
        Gh = O.ghat(g, p, Q, 1e30)   # eps huge: only -(1/tau){B:sigma + C.grad T} M remains
        i, j = n // 4, 3 * n // 8    # the cell centred at (0.25 + dx/2, 0.25 + dy/2)
        xc, yc = g.xc()[i], g.yc()[j]
        h = 1e-5
        v1, v2 = g.v1()[None, :], g.v2()[:, None]

        def M_at(xx, yy):
            r, a, b, t = _fields(xx, yy)
            return r / (2 * np.pi * t) * np.exp(-((v1 - a) ** 2 + (v2 - b) ** 2) / (2 * t))

        dMx = (M_at(xc + h, yc) - M_at(xc - h, yc)) / (2 * h)
        dMy = (M_at(xc, yc + h) - M_at(xc, yc - h)) / (2 * h)
        S = v1 * dMx + v2 * dMy
        r, a, b, t = _fields(xc, yc)
        ref = -(S - O.project(g, r, a, b, t, S))   # tau = 1
        errs.append(np.max(np.abs(Gh[j, i] - ref)) / np.max(np.abs(ref)))
    assert errs[-1] < 5e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0   # second order in dx


# ---------------------------------------------------------------------------------------------
# invariants of the whole step
# ---------------------------------------------------------------------------------------------
def _totals(Q):
    return np.array([Q[0].sum(), Q[1].sum(), Q[2].sum(), (Q[3] + Q[5]).sum()])


def test_conservation_periodic():
    g = I.Grid(nx=12, ny=10, nv1=16, nv2=16)
    p = I.Params(nu=-0.5, bc=(I.PERIODIC,) * 4)
    Q0 = I.smooth_state(g, seed=11)
    G0 = I.seeded_g(g, seed=12, amp=0.02)
    dt = O.dt_for_cfl(g, 0.5, 0.0, I.CFL_SUM)[0]
    for eps in (1e-3, 1e-1, 10.0):
        Q, G, H = O.step(g, p, Q0, G0, dt, eps, 40)
        t0, t1 = _totals(Q0), _totals(Q)
        scale = np.array([t0[0], t0[0], t0[0], t0[3]])
        assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (eps, t1 - t0)


def test_specular_conserves_mass_and_energy():
    g = I.Grid(nx=10, ny=12, nv1=16, nv2=16)
    p = I.Params(nu=-0.5, bc=(I.SPECULAR,) * 4)
    Q0 = I.smooth_state(g, seed=21, umax=0.2)
    dt = O.dt_for_cfl(g, 0.5, 0.0, I.CFL_SUM)[0]
    Q, G, H = O.step(g, p, Q0, I.zero_g(g), dt, 1e-2, 40)
    t0, t1 = _totals(Q0), _totals(Q)
    assert abs(t1[0] - t0[0]) <= 1e-13 * t0[0]
    assert abs(t1[3] - t0[3]) <= 1e-13 * t0[3]


def test_specular_mirror_symmetry():
    """A state symmetric about x = 1/2 (u1 odd, others even) stays symmetric."""
    g = I.Grid(nx=10, ny=6, nv1=12, nv2=12)
    p = I.Params(nu=-0.5, bc=(I.SPECULAR,) * 4)
    x, y = np.meshgrid(g.xc(), g.yc())
    rho = 1 + 0.3 * np.cos(2 * np.pi * x) + 0.1 * np.cos(np.pi * y)
    u1 = 0.2 * np.sin(2 * np.pi * x)
    Q0 = I.q_from_prims(rho, u1, 0.05 * np.cos(np.pi * y), 1.0)
    dt = O.dt_for_cfl(g, 0.5, 0.0, I.CFL_SUM)[0]
    Q, G, H = O.step(g, p, Q0, I.zero_g(g), dt, 1e-2, 20)
    sgn = np.array([1, -1, 1, 1, -1, 1])[:, None, None]
    assert np.max(np.abs(Q - sgn * Q[:, :, ::-1])) < 1e-12
    assert np.max(np.abs(G - G[:, ::-1, :, ::-1])) < 1e-12 * max(1e-300, np.max(np.abs(G)))


@pytest.mark.parametrize("axis", ["x", "y"])
def test_diffuse_walls_mirror_symmetry(axis):
    """Two equal diffuse walls facing each other (same temperature; the same tangential speed for
    walls normal to y, zero for walls normal to x) keep a mirror-symmetric state mirror-symmetric,
    with and without the ES term of the wall-cell Ghat: the two sides of the wall treatment
    (ghost Maxwellians, wall densities, upwind inflow, heat-flux faces) are mirror images of each
    other.  A sign or index error on one side breaks it."""
    g = I.Grid(nx=10, ny=8, nv1=12, nv2=12)
    x, y = np.meshgrid(g.xc(), g.yc())
    if axis == "x":
        bc, wT, wU = (I.DIFFUSE, I.DIFFUSE, I.PERIODIC, I.PERIODIC), (1.2, 1.2, 1, 1), (0, 0, 0, 0)
        rho = 1 + 0.3 * np.cos(2 * np.pi * x) + 0.1 * np.cos(2 * np.pi * y)
        u1, u2 = 0.2 * np.sin(2 * np.pi * x), 0.05 * np.cos(2 * np.pi * y)
        sgn = np.array([1, -1, 1, 1, -1, 1])[:, None, None]
        mirror = lambda a: a[..., ::-1]  # noqa: E731
        gmirror = lambda G: G[:, ::-1, :, ::-1]  # noqa: E731
    else:
        bc, wT, wU = (I.PERIODIC, I.PERIODIC, I.DIFFUSE, I.DIFFUSE), (1, 1, 0.9, 0.9), (0, 0, 0.2, 0.2)
        rho = 1 + 0.3 * np.cos(2 * np.pi * y) + 0.1 * np.cos(2 * np.pi * x)
        u1, u2 = 0.05 * np.cos(2 * np.pi * x), 0.2 * np.sin(2 * np.pi * y)
        sgn = np.array([1, 1, -1, 1, -1, 1])[:, None, None]
        mirror = lambda a: a[..., ::-1, :]  # noqa: E731
        gmirror = lambda G: G[::-1, :, ::-1, :]  # noqa: E731
    Q0 = I.q_from_prims(rho, u1, u2, 1.0)
    dt = O.dt_for_cfl(g, 0.5, 0.0, I.CFL_SUM)[0]
    for keep in (1, 0):
        p = I.Params(nu=-0.5, bc=bc, wall_T=wT, wall_U=wU, wall_keep_es_term=keep)
        Q, G, H = O.step(g, p, Q0, I.zero_g(g), dt, 1e-2, 12)
        assert np.max(np.abs(Q - sgn * mirror(Q))) < 1e-12, (axis, keep)
        assert np.max(np.abs(G - gmirror(G))) < 1e-11 * np.max(np.abs(G)), (axis, keep)


@pytest.mark.parametrize("bc,u", [((I.PERIODIC,) * 4, (0.4, -0.3)), ((I.SPECULAR,) * 4, (0.0, 0.0)),
                                  ((I.EXTRAP,) * 4, (0.3, 0.2)), ((I.DIFFUSE,) * 4, (0.0, 0.0))])
def test_global_maxwellian_is_preserved(bc, u):
    g = I.Grid(nx=6, ny=5, nv1=16, nv2=16)
    p = I.Params(nu=-0.5, bc=bc, wall_T=(0.8,) * 4)
    Q0 = I.q_from_prims(np.full((5, 6), 1.3), u[0], u[1], 0.8)
    dt = O.dt_for_cfl(g, 0.5, 0.0, I.CFL_SUM)[0]
    Q, G, H = O.step(g, p, Q0, I.zero_g(g), dt, 1e-2, 25)
    assert np.max(np.abs(Q - Q0)) < 1e-13
    assert np.max(np.abs(G)) < 1e-11


def test_null_space_moments_of_g_vanish():
    # v in [-10, 10]^2 so that the Gaussian tails beyond the mesh (the only source of
    # non-orthogonality of the analytic projector on the midpoint grid) are below round-off
    g = I.Grid(nx=8, ny=8, nv1=40, nv2=40, v1min=-10, v1max=10, v2min=-10, v2max=10)
    p = I.Params(nu=-0.5, bc=(I.PERIODIC,) * 4)
    Q0 = I.smooth_state(g, seed=31, umax=0.3)
    dt = O.dt_for_cfl(g, 0.5, 0.0, I.CFL_SUM)[0]
    Q, G, H = O.step(g, p, Q0, I.zero_g(g), dt, 5e-2, 10)
    v1, v2 = g.v1()[None, :], g.v2()[:, None]
    for w in (np.ones_like(v1 * v2), v1 + 0 * v2, v2 + 0 * v1, v1 ** 2 + v2 ** 2):
        mom = np.einsum("jikl,kl->ji", G, w) * 0.25
        assert np.max(np.abs(mom)) <= 1e-12 * np.max(np.abs(G))


def test_space_homogeneous_es_relaxation_closed_form():
    """Uniform rho, u, T with anisotropic P: P11 - P22 and P12 decay as W^(2N) exactly
    (discrete closed form), tr P is preserved, and W^(2N) approaches exp(-tau(1-nu) t / eps)
    with second order in dt (TR-BDF2)."""
    g = I.Grid(nx=4, ny=4, nv1=24, nv2=24)
    nu, eps, rho, T = -0.5, 0.05, 1.1, 1.0
    p = I.Params(nu=nu, bc=(I.PERIODIC,) * 4, tau_model=I.TAU_RHO, tau0=1.0)
    Q0 = I.q_from_prims(np.full((4, 4), rho), 0.0, 0.0, T, 0.2, -0.15)
    D0 = Q0[3] - Q0[5]
    errs = []
    for nsteps in (10, 20, 40):
        dt = 0.02 / nsteps
        Q, G, H = O.step(g, p, Q0, I.zero_g(g), dt, eps, nsteps)
        W = O.trbdf2_W(rho, nu, eps, dt)
        D = Q[3] - Q[5]
        assert np.max(np.abs(D - W ** (2 * nsteps) * D0)) < 1e-13
        assert np.max(np.abs(Q[4] - W ** (2 * nsteps) * Q0[4])) < 1e-13
        assert np.max(np.abs((Q[3] + Q[5]) - (Q0[3] + Q0[5]))) < 1e-13
        errs.append(abs(W ** (2 * nsteps) - math.exp(-rho * (1 - nu) * 0.02 / eps)))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_ap_limit_g_equals_ghat():
    """eps -> 0: one step gives G^{n+1} = Ghat^n (Eq. 5-98 limit)."""
    g = I.Grid(nx=8, ny=6, nv1=16, nv2=16)
    p = I.Params(nu=-0.5, bc=(I.PERIODIC,) * 4)
    Q0 = I.smooth_state(g, seed=41, aniso=0.0)
    dt = O.dt_for_cfl(g, 0.5, 0.0, I.CFL_SUM)[0]
    eps = 1e-13
    Gh = O.ghat(g, p, Q0, eps)
    Q, G, H = O.step(g, p, Q0, I.seeded_g(g, 42), dt, eps, 1)
    assert np.max(np.abs(G - Gh)) <= 1e-7 * np.max(np.abs(Gh))


def test_free_streaming_limit_converges():
    """eps = 1e30: collisions vanish; the density of f = M + eps g follows the collisionless
    solution of a Maxwellian with sinusoidal density, rho(x,t) = 1 + A sin(2 pi x) exp(-2 pi^2 T t^2),
    with first-order convergence in dx."""
    A, T, tf = 0.2, 1.0, 0.1
    errs = []
    for nx in (25, 50, 100):
        g = I.Grid(nx=nx, ny=1, nv1=32, nv2=8)
        p = I.Params(nu=-0.5, bc=(I.PERIODIC,) * 4)
        x = g.xc()
        Q0 = I.q_from_prims((1 + A * np.sin(2 * np.pi * x))[None, :], 0.0, 0.0, T)
        dt, n = O.dt_for_cfl(g, 0.5, tf, I.CFL_SUM)
        Q, G, H = O.step(g, p, Q0, I.zero_g(g), dt, 1e30, n)
        exact = 1 + A * np.sin(2 * np.pi * x) * math.exp(-2 * math.pi ** 2 * T * tf ** 2)
        errs.append(np.mean(np.abs(Q[0, 0] - exact)))
    assert errs[0] / errs[1] > 1.6 and errs[1] / errs[2] > 1.6
    assert errs[-1] < 2e-3


@pytest.mark.slow
def test_euler_limit_sod():
    """Small eps: the 1D-2V Sod density approaches the exact Euler Riemann solution (gamma = 2)."""
    from euler_exact import sample
    errs = []
    for eps in (1e-2, 1e-3, 1e-4):
        pr = I.sod_1d2v(eps=eps)
        Q, G, H = O.step(pr.grid, pr.params, pr.Q, pr.G, pr.dt, pr.eps, pr.nsteps)
        x = pr.grid.xc()
        ex = sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 2.0, (x - 0.5) / 0.2)
        errs.append(np.mean(np.abs(Q[0, 0] - ex[0])))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.02


def test_q_from_prim_printed_initial_states():
    """The conservative initial states printed for the cylindrical Sod problem (Section 6.2) and
    the lid-driven cavity (Section 6.3) follow from their primitive fields."""
    gold = json.load(open(os.path.join(GOLDEN, "initial_states.json")))
    for case in gold["cases"]:
        rho, u1, u2, T = (np.array([v]) for v in case["prim"])
        Q = O.q_from_prim(rho, u1, u2, T)[:, 0]
        assert np.array_equal(Q, np.array(case["Q"])), case["name"]


def test_q_from_prim_round_trip_and_energy():
    """Q from (rho, u, T) gives back rho, u, T, an isotropic pressure tensor rho T I and the energy
    (1/2) tr E = (1/2) rho (|u|^2 + 2 T) of Section 2 (d_v = 2); a swapped or dropped term in any
    component breaks one of them."""
    rng = np.random.default_rng(5)
    n = 64
    rho = rng.uniform(0.1, 3.0, n)
    u1, u2 = rng.uniform(-2.0, 2.0, n), rng.uniform(-2.0, 2.0, n)
    T = rng.uniform(0.2, 4.0, n)
    Q = O.q_from_prim(rho, u1, u2, T)
    p = I.Params()
    for c in range(n):
        out = O.prims(p, Q[:, c])
        assert np.allclose(out[:4], [rho[c], u1[c], u2[c], T[c]], rtol=1e-13, atol=1e-13)
        P = rho[c] * T[c]
        assert np.allclose(out[4:7], [P, 0.0, P], rtol=1e-12, atol=1e-12 * P)
    energy = 0.5 * (Q[3] + Q[5])
    assert np.allclose(energy, 0.5 * rho * (u1 ** 2 + u2 ** 2 + 2.0 * T), rtol=1e-14)


@pytest.mark.parametrize("bad", ["rho", "T", "u"])
def test_q_from_prim_rejects_non_physical(bad):
    rho, u1, u2, T = (np.ones(3) for _ in range(4))
    if bad == "rho":
        rho[1] = 0.0
    elif bad == "T":
        T[2] = -1.0
    else:
        u1[0] = np.nan
    with pytest.raises(O.OracleError):
        O.q_from_prim(rho, u1, u2, T)


# ---------------------------------------------------------------------------------------------
# free streaming along y and along a diagonal of a mesh with dx != dy: fixes the transport
# scale of the y sweeps (micro, macro and heat-flux differences), which no x-only pin sees
# ---------------------------------------------------------------------------------------------
def _collisionless(k, T, A, X, Y, t, v1, v2):
    """Moments of f(x, v, t) = rho0(x - v t) M_T(v), rho0 = 1 + A sin(2 pi k.x), u = 0: with
    a = 2 pi k t and D = exp(-T |a|^2 / 2) (the characteristic function of the Gaussian),
    rho = 1 + A s D, m = -A c T a D, E = T I + A s (T I - T^2 a a^T) D (s, c the sine and cosine of
    2 pi k.x); and f itself at the cell centres and velocity nodes."""
    a = 2 * math.pi * np.array(k, dtype=float) * t
    D = math.exp(-T * (a @ a) / 2)
    ph = 2 * math.pi * (k[0] * X + k[1] * Y)
    s, c = np.sin(ph), np.cos(ph)
    Q = np.array([1 + A * s * D, -A * c * T * a[0] * D, -A * c * T * a[1] * D,
                  T + A * s * (T - T * T * a[0] * a[0]) * D, A * s * (-T * T * a[0] * a[1]) * D,
                  T + A * s * (T - T * T * a[1] * a[1]) * D])
    V1, V2 = v1[None, None, None, :], v2[None, None, :, None]
    ph2 = 2 * math.pi * (k[0] * (X[:, :, None, None] - V1 * t) + k[1] * (Y[:, :, None, None] - V2 * t))
    f = (1 + A * np.sin(ph2)) * np.exp(-(V1 ** 2 + V2 ** 2) / (2 * T)) / (2 * math.pi * T)
    return Q, f


def _free_stream_errors(nx, ny, k, nv, tf=0.1, A=0.2, T=1.0, eps=1e30):
    g = I.Grid(nx=nx, ny=ny, nv1=nv[0], nv2=nv[1])
    p = I.Params(nu=-0.5, bc=(I.PERIODIC,) * 4)
    X, Y = np.meshgrid(g.xc(), g.yc())
    Q0 = I.q_from_prims(1 + A * np.sin(2 * math.pi * (k[0] * X + k[1] * Y)), 0.0, 0.0, T)
    dt, n = O.dt_for_cfl(g, 0.5, tf, I.CFL_SUM)
    Q, G, H = O.step(g, p, Q0, I.zero_g(g), dt, eps, n)
    Qe, fe = _collisionless(k, T, A, X, Y, n * dt, g.v1(), g.v2())
    # the kinetic solution f_h = M[Q] + eps g, M from the moments of Q (u, T of the cell)
    rho = Q[0]
    u1, u2 = Q[1] / rho, Q[2] / rho
    Tn = (Q[3] + Q[5] - rho * (u1 * u1 + u2 * u2)) / (2 * rho)
    V1, V2 = g.v1()[None, None, None, :], g.v2()[None, None, :, None]
    w = lambda a: a[:, :, None, None]  # noqa: E731
    M = w(rho / (2 * math.pi * Tn)) * np.exp(-((V1 - w(u1)) ** 2 + (V2 - w(u2)) ** 2) / (2 * w(Tn)))
    eq = np.mean(np.abs(Q - Qe), axis=(1, 2))
    ef = np.mean(np.abs(M + eps * G - fe)) / np.mean(np.abs(fe))
    return eq, ef


def _assert_first_order(levels, comps):
    for (qa, fa), (qb, fb) in zip(levels, levels[1:]):
        assert fa / fb > 1.5, (fa, fb)
        for m in comps:
            assert qa[m] / qb[m] > 1.5, (m, qa[m], qb[m])


def test_free_streaming_along_y():
    """eps = 1e30 on a single column (nx = 1, dx = 1 != dy): density, y momentum, both normal
    energies and the kinetic solution f_h = M + eps g follow the collisionless solution with
    first-order convergence; a y transport scaled by dx instead of dy breaks it."""
    levels = [_free_stream_errors(1, ny, (0, 1), (8, 32)) for ny in (25, 50, 100)]
    _assert_first_order(levels, (0, 2, 3, 5))
    q, f = levels[-1]
    assert np.all(q[[0, 2, 3, 5]] < 2.5e-3) and f < 3e-3, (q, f)
    assert q[1] < 1e-15 and q[4] < 1e-15     # no x motion arises


def test_free_streaming_diagonal_unequal_cells():
    """eps = 1e30, density wave along (1, 1) on meshes with dy = (2/3) dx: all six moments and f_h
    converge at first order to the collisionless solution."""
    levels = [_free_stream_errors(n, 3 * n // 2, (1, 1), (16, 16)) for n in (12, 24, 48)]
    _assert_first_order(levels, range(6))
    q, f = levels[-1]
    assert np.all(q < 5e-3) and f < 8e-3, (q, f)


# ---------------------------------------------------------------------------------------------
# diffuse walls (Section 6.3): one step from a uniform gas at rest with an anisotropic diagonal
# pressure tensor next to a moving wall of another temperature, in closed form
# ---------------------------------------------------------------------------------------------
def _half_moments(r, theta_n, mu_t, theta_t, s):
    """r int_{s v_n > 0} v_n m(v) N(v_n; 0, theta_n) N(v_t; mu_t, theta_t) dv for the monomials
    m = (1, v_n, v_t, v_n^2, v_n v_t, v_t^2): half-line Gaussian moments times full-line ones."""
    i1, i2, i3 = s * math.sqrt(theta_n / (2 * math.pi)), theta_n / 2, s * 2 * theta_n * math.sqrt(theta_n / (2 * math.pi))
    j1, j2 = mu_t, mu_t * mu_t + theta_t
    return r * np.array([i1, i2, i1 * j1, i3, i2 * j1, i1 * j2])


def _to_q_order(F, d):
    """(1, v_n, v_t, v_n^2, v_n v_t, v_t^2) -> (1, v1, v2, v1^2, v1 v2, v2^2) for normal axis d."""
    if d == 0:
        return F
    return np.array([F[0], F[2], F[1], F[5], F[4], F[3]])


def _relax_half(q, W):
    """Collision half step of the ES-BGK macro equations: the trace of P is kept and its
    deviator is multiplied by W, the TR-BDF2 stability factor of y' = -tau (1 - nu) y / eps."""
    rho, m1, m2 = q[0], q[1], q[2]
    P = np.array([[q[3] - m1 * m1 / rho, q[4] - m1 * m2 / rho],
                  [q[4] - m1 * m2 / rho, q[5] - m2 * m2 / rho]])
    p = np.trace(P) / 2
    Pn = p * np.eye(2) + W * (P - p * np.eye(2))
    return np.array([rho, m1, m2, m1 * m1 / rho + Pn[0, 0], m1 * m2 / rho + Pn[0, 1],
                     m2 * m2 / rho + Pn[1, 1]])


def _wall_case(side, shear=0.0):
    d = side // 2                  # normal axis
    n_norm, n_tan = 4, 3
    nx, ny = (n_norm, n_tan) if d == 0 else (n_tan, n_norm)
    # cells of 0.1 along the wall normal, 0.1 along the wall; v in [-10, 10]^2 so that the
    # Gaussian tails beyond the mesh are below round-off
    g = I.Grid(nx=nx, ny=ny, x0=0, x1=0.1 * nx, y0=0, y1=0.1 * ny,
               nv1=40, nv2=40, v1min=-10, v1max=10, v2min=-10, v2max=10)
    bc = [I.PERIODIC] * 4
    bc[2 * d] = bc[2 * d + 1] = I.EXTRAP
    bc[side] = I.DIFFUSE
    wT, wU = [1.0] * 4, [0.0] * 4
    wT[side], wU[side] = 1.4, 0.35
    p = I.Params(nu=-0.5, bc=tuple(bc), wall_T=tuple(wT), wall_U=tuple(wU), tau_model=I.TAU_RHO,
                 tau0=1.0, wall_keep_es_term=1)
    rho, T, aniso = 1.3, 1.0, 0.15
    Q0 = I.q_from_prims(np.full((ny, nx), rho), 0.0, 0.0, T, aniso, shear)
    h = (g.x1 - g.x0) / nx if d == 0 else (g.y1 - g.y0) / ny
    cell = (slice(None), 0 if side == 2 else (ny - 1 if side == 3 else slice(None)),
            0 if side == 0 else (nx - 1 if side == 1 else slice(None)))
    return g, p, Q0, d, h, cell, rho, 1.4, 0.35


@pytest.mark.parametrize("side", [0, 1, 2, 3])
def test_diffuse_wall_macro_step_closed_form(side):
    """After one step from a uniform gas at rest (g = 0, P diagonal and anisotropic) the wall cell
    holds, to round-off, Q* = the first collision half step, plus dt/h times the net KFVS flux:
    through the wall, the wall-side half flux of the wall Maxwellian (density r_w from zero mass
    flux, r_w sqrt(T_w / 2 pi) = rho sqrt(T*_nn / 2 pi) with T*_nn of Q*, tangential velocity U,
    temperature T_w) plus the cell's own outgoing half flux; through the inner face, the full flux
    of the uniform state.  The heat-flux differences cancel in the wall cell (its inner neighbour
    has no third moments), and the last collision half step relaxes the result.  Pins the ghost
    state's orientation, velocity and density, and the split stage it is taken from."""
    g, p, Q0, d, h, cell, rho, Tw, U = _wall_case(side)
    eps, dt = 0.05, 2e-3
    Q, G, H = O.step(g, p, Q0, I.zero_g(g), dt, eps, 1)
    tau = rho                                         # tau = tau0 rho, rho unchanged (zero mass flux)
    W = _trbdf2_scalar(tau * (1 - p.nu) / eps, dt / 2)
    q0 = Q0[:, 0, 0]
    qs = _relax_half(q0, W)                           # Q*
    Tnn = (qs[3] if d == 0 else qs[5]) / rho
    Ttt = (qs[5] if d == 0 else qs[3]) / rho
    rw = rho * math.sqrt(Tnn / Tw)
    low = side % 2 == 0
    s_in = 1 if low else -1                           # the wall emits velocities pointing inward
    F_wall = (_half_moments(rw, Tw, U, Tw, s_in) + _half_moments(rho, Tnn, 0.0, Ttt, -s_in))
    F_wall = _to_q_order(F_wall, d)
    F_int = np.zeros(6)
    F_int[1 + d] = rho * Tnn                          # full flux of the uniform state at rest
    net = (F_wall - F_int) if low else (F_int - F_wall)
    want = _relax_half(qs + dt / h * net, W)
    got = Q[cell]
    got = got.reshape(6, -1)
    assert np.all(np.abs(got - want[:, None]) <= 1e-13 * max(1.0, np.max(np.abs(want)))), (got[:, 0], want)
    # the tangential momentum the moving wall hands to the gas: dt/h r_w U sqrt(T_w / 2 pi)
    assert abs(got[2 - d, 0] - dt / h * rw * U * math.sqrt(Tw / (2 * math.pi))) < 1e-14


@pytest.mark.parametrize("side", [0, 1, 2, 3])
@pytest.mark.parametrize("keep", [1, 0])
def test_diffuse_wall_micro_shear_closed_form(side, keep):
    """g after one step from g = 0 in the wall cell is (dt tau/(eps + dt tau)) Ghat_wall; its shear
    moment eps dv^2 sum v1 v2 g is, to round-off, w2 (+-(eps/tau) r_w U T_w / (2 h) + nu P12): the
    upwind difference against the wall Maxwellian (r_w from the time-n state's normal temperature,
    tangential velocity U) seen through (I - Pi_M), whose shear moment it keeps, plus the ES term
    eps (Gcal - M)/eps with shear moment nu P12 (dropped in the literal wall form)."""
    g, p, Q0, d, h, cell, rho, Tw, U = _wall_case(side, shear=0.1)
    p.wall_keep_es_term = keep
    eps, dt = 0.05, 2e-3
    Q, G, H = O.step(g, p, Q0, I.zero_g(g), dt, eps, 1)
    tau = rho
    w2 = dt * tau / (eps + dt * tau)
    P = np.array([[Q0[3, 0, 0], Q0[4, 0, 0]], [Q0[4, 0, 0], Q0[5, 0, 0]]])
    rw = rho * math.sqrt(P[d, d] / rho / Tw)
    sgn = 1 if side % 2 == 0 else -1
    want = w2 * (sgn * (eps / tau) * rw * U * Tw / (2 * h) + keep * p.nu * P[0, 1])
    V1, V2 = np.meshgrid(g.v1(), g.v2())
    dv2 = (g.v1()[1] - g.v1()[0]) * (g.v2()[1] - g.v2()[0])
    Gc = G[cell[1], cell[2]].reshape(-1, g.nv2, g.nv1)
    got = eps * dv2 * np.einsum("ckl,kl->c", Gc, V1 * V2)
    assert np.all(np.abs(got - want) <= 1e-12 * abs(want)), (got, want)


def test_diffuse_walls_conserve_mass():
    """Zero mass flux through every diffuse wall (wall densities of Section 6.3): with four moving
    walls of different temperatures and a flowing, anisotropic gas the total mass stays constant
    to round-off over many steps, while the energy does not (the walls exchange heat)."""
    g = I.Grid(nx=10, ny=9, nv1=16, nv2=16)
    p = I.Params(nu=-0.5, bc=(I.DIFFUSE,) * 4, wall_T=(1.3, 0.8, 1.1, 0.9),
                 wall_U=(0.2, -0.3, 0.25, -0.15))
    x, y = np.meshgrid(g.xc(), g.yc())
    rho = 1 + 0.3 * np.cos(2 * np.pi * x) * np.sin(np.pi * y) + 0.1 * x
    u1 = 0.3 * np.sin(2 * np.pi * y) + 0.2 * (x - 0.5)
    u2 = -0.25 * np.cos(np.pi * x) - 0.2 * (y - 0.5)
    Q0 = I.q_from_prims(rho, u1, u2, 1.0 + 0.2 * x * y, 0.1, -0.05)
    dt = O.dt_for_cfl(g, 0.5, 0.0, I.CFL_SUM)[0]
    for eps in (1e-2, 1.0):
        Q, G, H = O.step(g, p, Q0, I.zero_g(g), dt, eps, 30)
        assert abs(Q[0].sum() - Q0[0].sum()) <= 1e-13 * Q0[0].sum()
        assert abs((Q[3] + Q[5]).sum() - (Q0[3] + Q0[5]).sum()) > 1e-6
