"""The manufactured-solution harness on the GPU (Section 6.1, Table tab5-4): exact state, source
steps and error norms against the oracle, and the convergence study on the paper's meshes."""
import json
import math
import os

import numpy as np
import pytest

from helpers import q_rel_err
from oracle import oracle as O
from paper_2509_21832_gb300 import api
from paper_2509_21832_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mms_2d.json")
EPS = 0.08
ULP = 2.220446049250313e-16


def _case(nx, ny, nv1, nv2):
    g = I.Grid(nx=nx, ny=ny, nv1=nv1, nv2=nv2, v1min=-6, v1max=6, v2min=-6, v2max=6)
    p = I.Params(nu=-1.0, tau_model=I.TAU_HARDSPHERE2D, bc=(I.PERIODIC,) * 4)
    return g, p


def test_exact_state_and_source_steps_match_the_oracle():
    g, p = _case(12, 10, 16, 20)
    t0 = 0.1
    dt, _ = O.dt_for_cfl(g, 0.35, 0.25, I.CFL_SUM)
    with api.Solver(g, p) as s:
        s.mms_set_exact(t0, EPS)
        s.sync()
        Qg0, _ = s.get_moments()
        Gg0 = s.get_g()
        Qo0, Go0 = O.mms_exact(g, p, t0, EPS)
        assert np.max(np.abs(Qg0 - Qo0)) <= 1e-14 * np.max(np.abs(Qo0))
        assert np.max(np.abs(Gg0 - Go0)) <= 1e-13 * np.max(np.abs(Go0))
        s.mms_enable(True, t0)
        s.step(dt, EPS, 5)
        s.sync()
        Qg, Hg = s.get_moments()
        Gg = s.get_g()
        em, eu = s.mms_error(t0 + 5 * dt, EPS)
    Qo, Go, Ho = O.step_mms(g, p, Qo0, Go0, dt, EPS, 5, t0)
    assert np.all(q_rel_err(Qg, Qo) <= 1e-12), q_rel_err(Qg, Qo)
    gfl = 64 * ULP * np.max(Qo[0]) / EPS
    assert np.max(np.abs(Gg - Go)) <= max(1e-11 * np.max(np.abs(Go)), gfl)
    assert np.max(np.abs(Hg - Ho)) <= max(1e-11 * np.max(np.abs(Ho)), 64 * ULP * 8 * np.max(Qo[0]))
    Qe, Ge = O.mms_exact(g, p, t0 + 5 * dt, EPS)
    assert abs(em - math.sqrt(np.sum((Qg - Qe) ** 2) / np.sum(Qe ** 2))) <= 1e-12
    assert abs(eu - math.sqrt(np.sum((Gg - Ge) ** 2) / np.sum(Ge ** 2))) <= 1e-12


def test_harness_rejects_unsuitable_contexts():
    g = I.Grid(nx=8, ny=8, nv1=8, nv2=8)
    with api.Solver(g, I.Params(bc=(I.SPECULAR,) * 4)) as s:
        with pytest.raises(api.MMError):
            s.mms_enable(True, 0.0)
    with api.Solver(g, I.Params(bc=(I.PERIODIC,) * 4, precision=I.PREC_G_FP32)) as s:
        with pytest.raises(api.MMError):
            s.mms_set_exact(0.0, EPS)


def run_study(n, lo=-1.0, hi=1.0):
    g = I.Grid(nx=n, ny=n, x0=lo, x1=hi, y0=lo, y1=hi, nv1=n, nv2=n, v1min=-6, v1max=6,
               v2min=-6, v2max=6)
    p = I.Params(nu=-1.0, tau_model=I.TAU_HARDSPHERE2D, bc=(I.PERIODIC,) * 4)
    dt, ns = O.dt_for_cfl(g, 0.35, 0.25, I.CFL_SUM)
    with api.Solver(g, p) as s:
        s.mms_set_exact(0.0, EPS)
        s.mms_enable(True, 0.0)
        s.step(dt, EPS, ns)
        s.sync()
        return s.mms_error(ns * dt, EPS)


def test_convergence_study_under_the_stated_domain():
    """Table tab5-4 on the paper's meshes 40^4, 80^4, 160^4, t = 0.25, CFL 0.35, under the
    readings taken from Section 6.1: the stated domain [0, 1]^2 and the tau of the exact state
    in S.  Under them the errors come out at about half the printed ones (0.53-0.65 times: each
    printed row is close to our next coarser mesh), with first-order convergence whose
    pre-asymptotic orders run ahead of the printed ones by about one mesh.  The same meshes on
    [-1, 1]^2, which is not the stated domain, are reported beside them: there the printed
    errors come out to 10 % at 40^4, 5 % at 80^4 and 2 % at 160^4 and the printed orders to 0.1,
    an observation about the paper's runs, not a reading the tests rely on."""
    with open(GOLDEN) as f:
        table = {r["n"]: r for r in json.load(f)["table_tab5_4"]}
    stated = {n: run_study(n, 0.0, 1.0) for n in (40, 80, 160)}
    other = {n: run_study(n) for n in (40, 80, 160)}
    for n in (40, 80, 160):
        (em, eu), (fm, fu) = stated[n], other[n]
        print("%d^4: [0,1]^2 macro %.6e (%.3f of printed) micro %.6e (%.3f) | "
              "[-1,1]^2 macro %.6e (%.3f) micro %.6e (%.3f)"
              % (n, em, em / table[n]["macro"], eu, eu / table[n]["micro"],
                 fm, fm / table[n]["macro"], fu, fu / table[n]["micro"]))
        assert 0.45 <= em / table[n]["macro"] <= 0.75
        assert 0.45 <= eu / table[n]["micro"] <= 0.75
        tol = {40: 0.10, 80: 0.05, 160: 0.02}[n]
        assert abs(fm / table[n]["macro"] - 1) <= tol
        assert abs(fu / table[n]["micro"] - 1) <= tol
    for a, b in ((40, 80), (80, 160)):
        rm = math.log2(stated[a][0] / stated[b][0])
        ru = math.log2(stated[a][1] / stated[b][1])
        print("%d -> %d on [0,1]^2: orders %.3f (paper %.3f), %.3f (paper %.3f)"
              % (a, b, rm, table[b]["macro_rate"], ru, table[b]["micro_rate"]))
        assert 0.6 <= rm <= 1.05 and 0.6 <= ru <= 1.05
        assert rm >= table[b]["macro_rate"] - 0.05 and ru >= table[b]["micro_rate"] - 0.05
        fm = math.log2(other[a][0] / other[b][0])
        fu = math.log2(other[a][1] / other[b][1])
        assert abs(fm - table[b]["macro_rate"]) <= 0.1
        assert abs(fu - table[b]["micro_rate"]) <= 0.1
