"""The paper's lid-driven cavity (Section 6.3 example) at its production size, 240^2 x 14^2,
eps = 0.08, to t = 3 with CFL 0.95, as a diffuse-wall run through the C ABI: mass is conserved,
the flow settles to a steady state with the clockwise circulation the paper shows, and part of
the heat flows from cold to hot (the anti-Fourier heat flow the paper reports)."""
import numpy as np
import pytest

from paper_2509_21832_gb300 import api
from paper_2509_21832_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_lid_driven_cavity_production_run():
    g = I.Grid(nx=240, ny=240, nv1=14, nv2=14, v1min=-5, v1max=5, v2min=-5, v2max=5)
    p = I.Params(nu=-1.0, tau_model=I.TAU_HARDSPHERE2D, bc=(I.DIFFUSE,) * 4,
                 wall_T=(1.0,) * 4, wall_U=(0.0, 0.0, 0.0, 0.16))
    eps = 0.08
    dt, nsteps = api.mm_dt_for_cfl(g, 0.95, 3.0, I.CFL_SUM)
    one = np.ones((g.ny, g.nx))
    Q0 = I.q_from_prims(one, 0 * one, 0 * one, one)
    with api.Solver(g, p) as s:
        s.set_state(Q0, None)
        s.step(dt, eps, nsteps - 100)
        Qa, _ = s.get_moments(with_H=False)
        s.step(dt, eps, 100)
        Q, H = s.get_moments()
    mass0 = Q0[0].sum()
    assert abs(Q[0].sum() - mass0) <= 1e-12 * mass0
    # steady state: the last 100 steps (0.04 time units) change Q very little
    assert np.max(np.abs(Q - Qa)) <= 1e-3 * np.max(np.abs(Q))
    rho = Q[0]
    u1, u2 = Q[1] / rho, Q[2] / rho
    n = g.nx
    # clockwise circulation under a lid moving right: right along the top, down the right wall,
    # left along the bottom, up the left wall
    assert u1[3 * n // 4:, :].mean() > 0 and u1[: n // 2, :].mean() < 0
    assert u2[:, 3 * n // 4:].mean() < 0 and u2[:, : n // 4].mean() > 0
    assert 0.0 < np.max(np.abs(u1)) < 0.16
    # heat flux h = (H111 + H122, H112 + H222) / 2 against -grad T
    T = (Q[3] + Q[5] - rho * (u1 ** 2 + u2 ** 2)) / (2 * rho)
    h1, h2 = 0.5 * (H[0] + H[2]), 0.5 * (H[1] + H[3])
    Ty, Tx = np.gradient(T, 1.0 / n, 1.0 / n)
    inner = (slice(10, n - 10), slice(10, n - 10))
    dot = (h1 * -Tx + h2 * -Ty)[inner]
    big = np.hypot(h1, h2)[inner] > 0.05 * np.max(np.hypot(h1, h2)[inner])
    anti = np.mean(dot[big] < 0)
    print("steps %d, max |u1| %.4f, T in [%.4f, %.4f], anti-Fourier fraction %.3f"
          % (nsteps, np.max(np.abs(u1)), T.min(), T.max(), anti))
    assert anti > 0.05
