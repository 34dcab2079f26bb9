"""Batched stepping (mm_batch_*): every problem of a mixed batch against the oracle, CUDA-graph
replay against direct launches, and the autotuner leaving the state untouched."""
import numpy as np
import pytest

from helpers import q_rel_err
from oracle import oracle as O
from paper_2509_21832_gb300 import api
from paper_2509_21832_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ULP = 2.220446049250313e-16


def mixed_batch():
    probs = [
        (I.Grid(nx=13, ny=11, nv1=24, nv2=24), I.Params(bc=(I.PERIODIC,) * 4), 1e-2),
        (I.Grid(nx=9, ny=14, nv1=16, nv2=16), I.Params(bc=(I.EXTRAP,) * 4), 0.3),
        (I.Grid(nx=10, ny=7, nv1=32, nv2=32), I.Params(bc=(I.SPECULAR,) * 4), 1e-3),
        (I.Grid(nx=8, ny=9, nv1=20, nv2=20, v1min=-5, v1max=5, v2min=-5, v2max=5),
         I.Params(bc=(I.DIFFUSE,) * 4, wall_U=(0, 0, 0, 0.16), nu=-1.0,
                  tau_model=I.TAU_HARDSPHERE2D), 0.08),
        (I.Grid(nx=6, ny=5, nv1=17, nv2=15, v1min=-6, v1max=6, v2min=-6, v2max=6),
         I.Params(bc=(I.PERIODIC, I.PERIODIC, I.SPECULAR, I.DIFFUSE), nu=0.3,
                  tau_model=I.TAU_PRESSURE), 1.0),
        (I.Grid(nx=40, ny=1, nv1=24, nv2=24), I.Params(bc=(I.EXTRAP, I.EXTRAP, I.PERIODIC, I.PERIODIC)), 1e-2),
    ]
    out = []
    for q, (g, p, eps) in enumerate(probs):
        Q = I.smooth_state(g, seed=100 + q, umax=0.2, aniso=0.06)
        G = I.seeded_g(g, seed=200 + q, amp=0.02)
        dt = O.dt_for_cfl(g, 0.5, 0.0, I.CFL_SUM)[0]
        out.append((g, p, eps, Q, G, dt))
    return out


def run_batch(probs, nsteps, graph=True, tune=False):
    with api.BatchSolver([p[0] for p in probs], [p[1] for p in probs]) as b:
        b.set_graph(graph)
        for q, (g, p, eps, Q, G, dt) in enumerate(probs):
            b.set_state(q, Q, G)
        dts = [p[5] for p in probs]
        epss = [p[2] for p in probs]
        if tune:
            b.step(dts, epss, 1)
            for q, (g, p, eps, Q, G, dt) in enumerate(probs):
                b.set_state(q, Q, G)
            b.autotune()
        b.step(dts, epss, nsteps)
        b.sync()
        return [b.get_moments(q) + (b.get_g(q),) for q in range(len(probs))]


def test_batch_matches_oracle_per_problem():
    probs = mixed_batch()
    res = run_batch(probs, 6)
    for (g, p, eps, Q, G, dt), (Qb, Hb, Gb) in zip(probs, res):
        Qo, Go, Ho = O.step(g, p, Q, G, dt, eps, 6)
        assert np.all(q_rel_err(Qb, Qo) <= 1e-12), (g, q_rel_err(Qb, Qo))
        rho = Qo[0]
        T = (Qo[3] + Qo[5] - (Qo[1] ** 2 + Qo[2] ** 2) / rho) / (2 * rho)
        gfloor = 64 * ULP * np.max(rho / (2 * np.pi * T)) / eps
        assert np.max(np.abs(Gb - Go)) <= max(1e-11 * np.max(np.abs(Go)), gfloor)
        hfloor = 64 * ULP * 4 * np.max(rho * T ** 1.5)
        assert np.max(np.abs(Hb - Ho)) <= max(1e-11 * np.max(np.abs(Ho)), hfloor)


def test_graph_replay_equals_direct_launches():
    probs = mixed_batch()
    a = run_batch(probs, 5, graph=True)
    b = run_batch(probs, 5, graph=False)
    for (Qa, Ha, Ga), (Qb, Hb, Gb) in zip(a, b):
        assert np.array_equal(Qa, Qb) and np.array_equal(Ga, Gb) and np.array_equal(Ha, Hb)


def test_autotune_keeps_state_and_results():
    probs = mixed_batch()
    tuned = run_batch(probs, 4, tune=True)
    for (g, p, eps, Q, G, dt), (Qb, Hb, Gb) in zip(probs, tuned):
        Qo, Go, Ho = O.step(g, p, Q, G, dt, eps, 4)
        assert np.all(q_rel_err(Qb, Qo) <= 1e-12)


def test_full_size_batch_matches_single_contexts():
    """The benchmark's batch (64 periodic problems of 64-256 cells per side, 16^2 ... 32^2
    velocity meshes, eps log-uniform on [1e-3, 1]; about 9.4e8 phase cells), autotuned as the
    benchmark runs it: after two steps every problem's Q, H and g equal those of a single-problem
    context bit for bit (the same device bodies run per cell; the single contexts are checked
    against the oracle at full size in tests/test_parity_gpu.py)."""
    probs = I.batch_problems(count=64, seed=0, nmin=64, nmax=256)
    dts = [p.dt for p in probs]
    epss = [p.eps for p in probs]
    with api.BatchSolver([p.grid for p in probs], [p.params for p in probs]) as b:
        for q, p in enumerate(probs):
            b.set_state(q, p.Q, None)
        b.step(dts, epss, 1)
        for q, p in enumerate(probs):
            b.set_state(q, p.Q, None)
        b.autotune()
        b.step(dts, epss, 2)
        b.sync()
        got = {}
        for q in range(0, len(probs), 7):  # every 7th problem: all mesh sizes and eps decades
            got[q] = b.get_moments(q) + (b.get_g(q),)
    for q, (Qb, Hb, Gb) in got.items():
        p = probs[q]
        with api.Solver(p.grid, p.params) as s:
            s.set_state(p.Q, None)
            s.step(p.dt, p.eps, 2)
            Qs, Hs = s.get_moments()
            Gs = s.get_g()
        assert np.array_equal(Qb, Qs) and np.array_equal(Hb, Hs) and np.array_equal(Gb, Gs), \
            (q, p.grid.nx, p.grid.ny, p.grid.nv1, p.eps)


def test_one_launch_for_many_steps_equals_launch_per_step():
    """A call of several steps is one persistent launch whose queue holds every step's items;
    its results equal those of one launch per step bit for bit (the queue only orders work)."""
    probs = mixed_batch()
    many = run_batch(probs, 5)
    with api.BatchSolver([p[0] for p in probs], [p[1] for p in probs]) as b:
        for q, (g, p, eps, Q, G, dt) in enumerate(probs):
            b.set_state(q, Q, G)
        for _ in range(5):
            b.step([p[5] for p in probs], [p[2] for p in probs], 1)
        b.sync()
        one = [b.get_moments(q) + (b.get_g(q),) for q in range(len(probs))]
    for (Qa, Ha, Ga), (Qb, Hb, Gb) in zip(many, one):
        assert np.array_equal(Qa, Qb) and np.array_equal(Ga, Gb) and np.array_equal(Ha, Hb)


@pytest.mark.parametrize("q,phase,nsteps", [(1, 2, 1), (3, 4, 1), (0, 7, 3)])
def test_bounded_wait_runs_out_and_reports_timeout(q, phase, nsteps):
    """A dependency that is never released (the completions of one phase of one problem are not
    counted) makes the items waiting on it give up after the wait bound: mm_batch_sync reports
    MM_ERR_TIMEOUT, the launch ends within a few wait bounds, no fault is raised, and after the
    state is set again the batch steps exactly as a fresh one.  Holding the last phase of a
    problem with three steps in the launch stalls the next step's first phases."""
    import time
    probs = mixed_batch()
    ref = run_batch(probs, 2)
    dts, epss = [p[5] for p in probs], [p[2] for p in probs]
    with api.BatchSolver([p[0] for p in probs], [p[1] for p in probs]) as b:
        for k, (g, p, eps, Q, G, dt) in enumerate(probs):
            b.set_state(k, Q, G)
        b.diag_hold(q, phase, 50.0)
        t0 = time.perf_counter()
        b.step(dts, epss, nsteps)
        with pytest.raises(api.MMError) as e:
            b.sync()
        assert e.value.status == api.MM_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 10.0
        b.diag_hold(-1, -1)
        for k, (g, p, eps, Q, G, dt) in enumerate(probs):
            b.set_state(k, Q, G)
        b.step(dts, epss, 2)
        b.sync()
        got = [b.get_moments(k) + (b.get_g(k),) for k in range(len(probs))]
    for (Qa, Ha, Ga), (Qb, Hb, Gb) in zip(ref, got):
        assert np.array_equal(Qa, Qb) and np.array_equal(Ga, Gb) and np.array_equal(Ha, Hb)


def test_autotuned_tiles_are_reported():
    probs = mixed_batch()
    with api.BatchSolver([p[0] for p in probs], [p[1] for p in probs]) as b:
        for k, (g, p, eps, Q, G, dt) in enumerate(probs):
            b.set_state(k, Q, G)
        b.step([p[5] for p in probs], [p[2] for p in probs], 1)
        threads, ctas = b.autotune()
        tm, tc = b.tiles()
        assert threads == 32 and ctas >= 152
        assert tm in (1, 2, 4, 8) and tc in (threads, 4 * threads)
