"""Pins of the oracle's manufactured-solution harness (Section 6.1, 2D2V method of manufactured
solutions): the exact moments and Maxwellian against the formulas printed in the paper
(tests/golden/mms_2d.json), the exact moments against quadrature of f, the residual source's
moments against the conservation-law residuals in closed form, and first-order convergence of
the scheme with the source."""
import json
import math
import os

import numpy as np

from oracle import oracle as O
from paper_2509_21832_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mms_2d.json")
EPS = 0.08


def _case(n, nv=None, vmax=6.0):
    nv = nv or n
    g = I.Grid(nx=n, ny=n, nv1=nv, nv2=nv, v1min=-vmax, v1max=vmax, v2min=-vmax, v2max=vmax)
    p = I.Params(nu=-1.0, tau_model=I.TAU_HARDSPHERE2D, bc=(I.PERIODIC,) * 4)
    return g, p


def _phi(v1, v2):
    return np.exp(-(v1 - 1) ** 2 - (v2 - 1) ** 2) + 2 * np.exp(-(v1 + 1) ** 2 - (v2 + 1) ** 2)


def test_exact_moments_and_maxwellian_match_the_printed_formulas():
    with open(GOLDEN) as f:
        fx = json.load(f)
    g, p = _case(6, nv=12)
    for t in (0.0, 0.13, 0.25):
        Q, G = O.mms_exact(g, p, t, EPS)
        x, y = np.meshgrid(g.xc(), g.yc())
        base = math.pi / 3 - (math.pi / 6) * np.cos(2 * np.pi * (t - y)) * np.sin(2 * np.pi * (t - x))
        c = fx["printed_moments"]["coeff"]
        rho, m1, m2 = Q[0], Q[1], Q[2]
        P = [Q[3] - m1 * m1 / rho, Q[4] - m1 * m2 / rho, Q[5] - m2 * m2 / rho]
        for got, k in zip([rho, m1, m2] + P, c):
            assert np.allclose(got, k * base, rtol=1e-13, atol=0)
        # g = (f - M)/eps with M as printed
        mx = fx["printed_maxwellian"]
        F = 2 - np.sin(2 * np.pi * (t - x)) * np.cos(2 * np.pi * (t - y))
        v1, v2 = np.meshgrid(g.v1(), g.v2())
        M = mx["prefactor"] * np.exp(-(mx["a"] * v1 + mx["b"]) ** 2 - (mx["a"] * v2 + mx["b"]) ** 2)
        f = _phi(v1, v2)
        ge = (f[None, None] - M[None, None]) * F[:, :, None, None] / EPS
        assert np.allclose(G, ge, rtol=0, atol=1e-13 * np.max(np.abs(ge)))


def test_exact_moments_equal_quadrature_of_f():
    g, p = _case(4)
    Q, _ = O.mms_exact(g, p, 0.07, EPS)
    xg, wg = np.polynomial.legendre.leggauss(80)
    v = 10.0 * xg
    w = 10.0 * wg
    V1, V2 = np.meshgrid(v, v)
    W = np.outer(w, w)
    ph = _phi(V1, V2)
    mom = [np.sum(W * ph * m) for m in (1, V1, V2, V1 * V1, V1 * V2, V2 * V2)]
    x, y = np.meshgrid(g.xc(), g.yc())
    F = 2 - np.sin(2 * np.pi * (0.07 - x)) * np.cos(2 * np.pi * (0.07 - y))
    for m in range(6):
        assert np.allclose(Q[m], mom[m] * F, rtol=1e-13)


def test_source_moments_are_the_conservation_residuals():
    # int (1, v) S = d/dt (rho, rho u) + div of the fluxes (the collision term conserves them);
    # int v (x) v S = d/dt E + div of the third moments - (tau/eps) rho (Tcal - Theta)
    g, p = _case(4, nv=96, vmax=9.0)
    dv = (18.0 / 96) ** 2
    V1, V2 = np.meshgrid(g.v1(), g.v2())
    for (t, x, y) in ((0.0, 0.1, 0.7), (0.2, 0.45, 0.3)):
        S = O.mms_source(g, p, EPS, t, x, y)
        w = 2 * np.pi
        s1, c1 = np.sin(w * (t - x)), np.cos(w * (t - x))
        s2, c2 = np.sin(w * (t - y)), np.cos(w * (t - y))
        F = 2 - s1 * c2
        Ft, Fx, Fy = -w * c1 * c2 + w * s1 * s2, w * c1 * c2, -w * s1 * s2
        pi = np.pi
        # moments of phi: mass 3 pi, first (-pi, -pi), second E = pi (4.5, 3, 4.5); third
        # moments of a Gaussian of mean m and variance 1/2 per component:
        # m_i m_j m_k + (m_i d_jk + m_j d_ik + m_k d_ij)/2
        def third(i, j, k):
            tot = 0.0
            for mass, m in ((pi, (1.0, 1.0)), (2 * pi, (-1.0, -1.0))):
                d = lambda a, b: 1.0 if a == b else 0.0
                tot += mass * (m[i] * m[j] * m[k] + 0.5 * (m[i] * d(j, k) + m[j] * d(i, k) + m[k] * d(i, j)))
            return tot
        rho = 3 * pi * F
        E = {(0, 0): 4.5 * pi, (0, 1): 3 * pi, (1, 1): 4.5 * pi}
        tau = 3 * pi * 0.436 * rho / (math.sqrt(2.0) * 2.0)
        T = 25.0 / 18.0
        Theta = np.array([[25 / 18, 8 / 9], [8 / 9, 25 / 18]])
        Tcal = 2.0 * T * np.eye(2) - Theta  # nu = -1
        want = [3 * pi * Ft - pi * Fx - pi * Fy,
                -pi * Ft + E[(0, 0)] * Fx + E[(0, 1)] * Fy,
                -pi * Ft + E[(0, 1)] * Fx + E[(1, 1)] * Fy]
        for (i, j) in ((0, 0), (0, 1), (1, 1)):
            coll = -(tau / EPS) * rho * (Tcal[i, j] - Theta[i, j])
            want.append(E[(i, j)] * Ft + third(i, j, 0) * Fx + third(i, j, 1) * Fy + coll)
        got = [np.sum(S * m) * dv for m in (1, V1, V2, V1 * V1, V1 * V2, V2 * V2)]
        scale = max(abs(a) for a in want)
        for a, b in zip(got, want):
            assert abs(a - b) <= 1e-10 * scale, (a, b)


def _errors(n):
    g, p = _case(n)
    dt, ns = O.dt_for_cfl(g, 0.35, 0.25, I.CFL_SUM)
    Q0, G0 = O.mms_exact(g, p, 0.0, EPS)
    Q, G, _ = O.step_mms(g, p, Q0, G0, dt, EPS, ns, 0.0)
    Qe, Ge = O.mms_exact(g, p, ns * dt, EPS)
    return (math.sqrt(np.sum((Q - Qe) ** 2) / np.sum(Qe ** 2)),
            math.sqrt(np.sum((G - Ge) ** 2) / np.sum(Ge ** 2)))


def test_scheme_with_source_converges():
    # pre-asymptotic first-order convergence on the coarse meshes the oracle affords (the GPU
    # test runs the paper's 40^4 .. 160^4 meshes)
    e16 = _errors(16)
    e32 = _errors(32)
    for a, b in zip(e16, e32):
        assert b < a / 1.35, (e16, e32)
    assert e32[0] < 0.1 and e32[1] < 0.2


def test_micro_part_stays_orthogonal_to_the_null_space_with_the_source():
    # the source enters Ghat projected by (I - Pi_M), so g keeps zero (1, v, |v|^2) moments
    g, p = _case(6, nv=40, vmax=10.0)
    dt, _ = O.dt_for_cfl(g, 0.35, 0.25, I.CFL_SUM)
    Q0, G0 = O.mms_exact(g, p, 0.0, EPS)
    _, G, _ = O.step_mms(g, p, Q0, G0, dt, EPS, 3, 0.0)
    V1, V2 = np.meshgrid(g.v1(), g.v2())
    scale = np.max(np.sum(np.abs(G), axis=(2, 3)))
    for m in (1, V1, V2, V1 * V1 + V2 * V2):
        assert np.max(np.abs(np.sum(G * m, axis=(2, 3)))) <= 1e-11 * scale * np.max(np.abs(m))


def _study_40(lo, hi):
    g = I.Grid(nx=40, ny=40, x0=lo, x1=hi, y0=lo, y1=hi, nv1=40, nv2=40, v1min=-6, v1max=6,
               v2min=-6, v2max=6)
    p = I.Params(nu=-1.0, tau_model=I.TAU_HARDSPHERE2D, bc=(I.PERIODIC,) * 4)
    dt, ns = O.dt_for_cfl(g, 0.35, 0.25, I.CFL_SUM)
    Q0, G0 = O.mms_exact(g, p, 0.0, EPS)
    Q, G, _ = O.step_mms(g, p, Q0, G0, dt, EPS, ns, 0.0)
    Qe, Ge = O.mms_exact(g, p, ns * dt, EPS)
    return (math.sqrt(np.sum((Q - Qe) ** 2) / np.sum(Qe ** 2)),
            math.sqrt(np.sum((G - Ge) ** 2) / np.sum(Ge ** 2)))


def test_coarsest_printed_row():
    """Table tab5-4, 40^4, under the readings taken from Section 6.1: the domain [0, 1]^2 that
    the caption and the text state, and the tau of the exact state in S (S is a function of
    (t, x, v) alone).  Under them the oracle's errors are 0.61 (macro) and 0.64 (micro) times
    the printed ones -- about the printed 80^4 row.  The same mesh on [-1, 1]^2, which is not
    the stated domain, is reported beside it: there the printed row comes out to 10 %."""
    with open(GOLDEN) as f:
        row = json.load(f)["table_tab5_4"][0]
    em, eu = _study_40(0.0, 1.0)
    print("[0,1]^2: macro %.4e (%.3f of printed), micro %.4e (%.3f)"
          % (em, em / row["macro"], eu, eu / row["micro"]))
    assert 0.5 <= em / row["macro"] <= 0.75, em
    assert 0.5 <= eu / row["micro"] <= 0.75, eu
    em2, eu2 = _study_40(-1.0, 1.0)
    print("[-1,1]^2: macro %.4e (%.3f of printed), micro %.4e (%.3f)"
          % (em2, em2 / row["macro"], eu2, eu2 / row["micro"]))
    assert abs(em2 / row["macro"] - 1) <= 0.10 and abs(eu2 / row["micro"] - 1) <= 0.10
