"""GPU tests of the learned closure through the C ABI: the network's forward pass, gradient and
Adam step against the FP64 CPU reference (same BF16 weights), the features and Chapman-Enskog
flux against the closure oracle, one hybrid step against the oracle's hybrid step, and the
trained network's gain over the plain method (speed at a stated density error)."""

import numpy as np
import pytest

from helpers import q_rel_err
from oracle import closure_oracle as C
from oracle import mlp_oracle as M
from oracle import oracle as O
from paper_2509_21832_gb300 import api
from paper_2509_21832_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ULP = 2.220446049250313e-16


def _torch():
    import torch
    return torch


def _norm(seed, ystd=1.0):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.standard_normal(39) * 0.1, np.exp(rng.uniform(-0.5, 0.5, 39)),
                           rng.standard_normal(4) * 0.1 * ystd,
                           ystd * np.exp(rng.uniform(-0.5, 0.5, 4))]).astype(np.float32)


def _data_norm(X, seed):
    """Normalisation standardising the features of a case (as a trained network's does), with
    outputs scaled to ~1e-6."""
    # spreads floored at 1e-3 |mean|, so that the FP32 rounding of a feature moves its
    # standardised value by at most ~6e-5
    sx = np.maximum(X.std(axis=0), 1e-3 * np.abs(X.mean(axis=0)))
    isx = np.where(sx > 1e-12, 1.0 / np.maximum(sx, 1e-12), 1.0)
    n = _norm(seed, ystd=1e-6)
    return np.concatenate([X.mean(axis=0), isx, n[78:]]).astype(np.float32)


def _params(seed):
    p = M.init_params(seed).astype(np.float64)
    rng = np.random.default_rng(seed + 1)
    p[M.OFF_B1:M.OFF_W2] = rng.standard_normal(64) * 0.1
    p[M.OFF_B2:M.OFF_W3] = rng.standard_normal(64) * 0.1
    p[M.OFF_B3:] = rng.standard_normal(4) * 0.1
    return p.astype(np.float32)


def test_mlp_forward_and_bf16_weights_match_oracle():
    torch = _torch()
    params, norm = _params(1), _norm(2)
    mlp = api.MLP(params, norm)
    master, wb = mlp.get_params()
    assert np.array_equal(master, params)
    assert np.array_equal(wb.astype(np.float64), M.bf16_round(params))  # RNE on both sides
    for n in (1, 127, 1000, 4099):
        X = (np.random.default_rng(n).standard_normal((n, 39)) * 1.3).astype(np.float32)
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        mlp.forward(Xd, Yd)
        Y = Yd.cpu().numpy().astype(np.float64)
        Yo = M.forward(M.bf16_round(params), norm.astype(np.float64), X.astype(np.float64))
        tol = 2e-5 * (1.0 + np.max(np.abs(Yo)))
        assert np.max(np.abs(Y - Yo)) <= tol, (n, np.max(np.abs(Y - Yo)), tol)
    mlp.close()


def test_mlp_gradient_matches_oracle():
    torch = _torch()
    params, norm = _params(3), _norm(4)
    mlp = api.MLP(params, norm)
    for n in (1, 333, 2048):
        rng = np.random.default_rng(10 + n)
        X = (rng.standard_normal((n, 39)) * 1.1).astype(np.float32)
        T = rng.standard_normal((n, 4)).astype(np.float32)
        L, g = mlp.grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
        # the kernels' products take BF16 operands (activations, back-propagated gradients) with
        # FP32 accumulation: the oracle rounds the same operands
        Lo, go = M.loss_and_grad_bf16(M.bf16_round(params), norm.astype(np.float64),
                                      X.astype(np.float64), T.astype(np.float64))
        assert abs(L - Lo) <= 2e-5 * Lo, (n, L, Lo)
        err = np.max(np.abs(g.astype(np.float64) - go))
        assert err <= 1e-4 * np.max(np.abs(go)), (n, err, np.max(np.abs(go)))
        # every layer's gradient (weights and biases) is checked, not only the largest
        for a, b in ((M.OFF_W1, M.OFF_B1), (M.OFF_B1, M.OFF_W2), (M.OFF_W2, M.OFF_B2),
                     (M.OFF_B2, M.OFF_W3), (M.OFF_W3, M.OFF_B3), (M.OFF_B3, M.N_PARAM)):
            e = np.max(np.abs(g[a:b] - go[a:b]))
            assert e <= 1e-4 * np.max(np.abs(go[a:b])) + 1e-9, (n, a, e)
        # and the BF16 operands cost no more than a few BF16 units against the plain gradient
        _, gx = M.loss_and_grad(M.bf16_round(params), norm.astype(np.float64),
                                X.astype(np.float64), T.astype(np.float64))
        assert np.max(np.abs(g - gx)) <= 2.0 ** -5 * np.max(np.abs(gx))
    mlp.close()


def test_adam_step_matches_oracle():
    torch = _torch()
    params, norm = _params(5), _norm(6)
    mlp = api.MLP(params, norm)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((900, 39)).astype(np.float32)
    T = rng.standard_normal((900, 4)).astype(np.float32)
    lr = 1e-3
    for t in (1, 2):
        Lo, go = M.loss_and_grad_bf16(M.bf16_round(params if t == 1 else w_gpu),
                                      norm.astype(np.float64), X.astype(np.float64),
                                      T.astype(np.float64))
        if t == 1:
            w_o, m1, m2 = M.adam_step(params.astype(np.float64), 0.0, 0.0, go, 1, lr)
        else:
            w_o, m1, m2 = M.adam_step(w_gpu.astype(np.float64), m1, m2, go, 2, lr)
        mlp.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), lr)
        w_gpu, wb = mlp.get_params()
        sel = np.abs(go) > 1e-2 * np.max(np.abs(go))  # where FP32 and FP64 gradients agree in sign
        err = np.abs(w_gpu.astype(np.float64) - w_o)[sel]
        assert np.all(err <= 1e-2 * lr + 2.0 ** -22 * np.abs(w_o[sel])), (t, err.max())
        assert np.array_equal(wb.astype(np.float64), M.bf16_round(w_gpu))
    mlp.close()


FEATURE_CASES = [
    ("periodic", (I.PERIODIC,) * 4),
    ("specular_extrap", (I.SPECULAR, I.EXTRAP, I.PERIODIC, I.PERIODIC)),
    ("walls", (I.EXTRAP, I.SPECULAR, I.SPECULAR, I.DIFFUSE)),
]


@pytest.mark.parametrize("name,bc", FEATURE_CASES)
def test_features_and_chapman_enskog_flux_match_oracle(name, bc):
    torch = _torch()
    g = I.Grid(nx=13, ny=11, nv1=8, nv2=8)
    p = I.Params(nu=-0.5, bc=bc, tau_model=I.TAU_PRESSURE)
    Q = I.smooth_state(g, 21, amp=0.25, umax=0.3, aniso=0.1)
    eps, dt = 2e-2, 1e-3
    X = torch.empty((g.ncell, 39), dtype=torch.float32, device="cuda")
    aux = torch.empty((5, g.ny, g.nx), dtype=torch.float64, device="cuda")
    with api.Solver(g, p) as s:
        s.set_state(Q)
        s.closure_features(dt, eps, X, aux)
        s.sync()
    Xo, Hce, scale = C.features(g, p, Q, eps, dt)
    Xg = X.cpu().numpy().astype(np.float64)
    # The neighbour differences are FP64 subtractions rounded once to FP32; the scalings and the
    # non-difference features are FP32 expressions of FP32-rounded fields.  Counting one rounding
    # of u = 2^-24 per FP32 operation and per rounded input: the Knudsen scale carries at most
    # 7.5 u, each scaled difference 12 u, every other feature at most 6 u; log10 k adds the
    # scale's 7.5 u / ln 10 absolute to the 2-ulp error of log10f.
    u = 2.0 ** -24
    tol = 16 * u * np.abs(Xo) + 1e-30
    tol[:, 38] += 4 * u
    assert np.all(np.abs(Xg - Xo) <= tol), (name, np.max(np.abs(Xg - Xo) / tol))
    A = aux.cpu().numpy()
    assert np.max(np.abs(A[:4] - Hce)) <= 1e-13 * np.max(np.abs(Hce)), name
    assert np.max(np.abs(A[4] - scale) / scale) <= 1e-15, name


def _gap_thresholds(ind, interior):
    """Thresholds in the gaps of the middle half of the sorted indicator values, widest gap
    first (relative width above 1e-3), so that FP32 and FP64 evaluations of the network decide
    every cell alike."""
    v = np.sort(ind[interior])
    lo, hi = len(v) // 4, 3 * len(v) // 4
    d = np.diff(v[lo:hi + 1])
    out = []
    for k in np.argsort(-d):
        thr = 0.5 * (v[lo + k] + v[lo + k + 1])
        if d[k] / thr > 1e-3:
            out.append(thr)
    return out


HYBRID_CASES = [
    ("specular_16", dict(nx=14, ny=12, nv1=16, nv2=16), (I.SPECULAR,) * 4, 1e-2),
    ("periodic_24", dict(nx=11, ny=13, nv1=24, nv2=24), (I.PERIODIC,) * 4, 1e-3),
    ("mixed_20", dict(nx=12, ny=10, nv1=20, nv2=20), (I.EXTRAP, I.EXTRAP, I.PERIODIC, I.PERIODIC), 1e-1),
]


@pytest.mark.parametrize("name,gk,bc,eps", HYBRID_CASES)
def test_hybrid_steps_match_oracle(name, gk, bc, eps):
    """Two hybrid steps (the second one refreshes the g its sweeps read) against the oracle.  The
    network's outputs are scaled to ~1e-6 so that the heat flux it contributes differs between
    the FP32 kernels and the FP64 reference far below the macro-field tolerance; the threshold
    sits in a gap of the indicator values of both steps."""
    g = I.Grid(**gk)
    p = I.Params(nu=-0.5, bc=bc)
    Q = I.smooth_state(g, 31, amp=0.2, umax=0.25, aniso=0.05)
    G0 = I.seeded_g(g, 32, amp=0.02)
    dt = 0.5 / (8.0 * g.nx + 8.0 * g.ny)
    X, _, _ = C.features(g, p, Q, eps, dt)
    params, norm = _params(8), _data_norm(X, 9)
    wq = M.bf16_round(params)
    net = lambda X: M.forward(wq, norm.astype(np.float64), X)
    interior = ~C.boundary_cells(g, p)
    ind0 = np.max(np.abs(net(X)), axis=1).reshape(g.ny, g.nx)
    ref = None
    for thr in _gap_thresholds(ind0, interior):
        Qo, Go, Ho, fo, io, ro = C.hybrid_run(g, p, Q, G0, dt, eps, net, thr, nsteps=2)
        sep = min(np.min(np.abs(i[interior] - thr)) for i in io) / thr
        if sep > 5e-4 and 0 < fo[1].sum() < interior.sum():
            ref = (thr, Qo, Go, Ho, fo, ro)
            break
    assert ref is not None
    thr, Qo, Go, Ho, fo, ro = ref
    assert ro[1].sum() > 0  # the second step refreshes cells
    mlp = api.MLP(params, norm)
    with api.Solver(g, p) as s:
        s.set_state(Q, G0)
        s.set_closure(mlp, thr)
        s.set_closure_fallback(0.0, 1)  # both steps hybrid, as in the oracle's run
        s.step(dt, eps, 2)
        s.sync()
        Qg, Hg = s.get_moments()
        Gg = s.get_g()
        fg = s.closure_flags().astype(bool)
        ncl, ncs = s.closure_stats()
    assert np.array_equal(fg, fo[1]), name
    assert ncl == fo[0].sum() + fo[1].sum() and ncs == 2 * g.ncell
    eq = q_rel_err(Qg, Qo)
    assert np.all(eq <= 1e-12), (name, eq)
    rho = np.asarray(Q).reshape(6, g.ny, g.nx)[0]
    gfl = 64 * ULP * np.max(rho) / eps
    gerr = np.max(np.abs(Gg - Go))
    assert gerr <= max(1e-11 * np.max(np.abs(Go)), gfl), (name, gerr)
    herr = np.max(np.abs(Hg - Ho))
    assert herr <= max(1e-11 * np.max(np.abs(Ho)), 64 * ULP * 8.0 * np.max(rho)), (name, herr)
    mlp.close()


def test_switching_the_closure_off_resets_stale_g():
    """After hybrid steps, switching the closure off and stepping is the oracle's plain step from
    the hybrid state with every non-current g reset to Ghat(Q^n)."""
    g = I.Grid(nx=12, ny=10, nv1=16, nv2=16)
    p = I.Params(nu=-0.5, bc=(I.SPECULAR,) * 4)
    Q = I.smooth_state(g, 51, amp=0.2, umax=0.25, aniso=0.05)
    G0 = I.seeded_g(g, 52, amp=0.02)
    dt, eps = 0.5 / (16.0 * 12 + 16.0 * 10), 1e-2
    X, _, _ = C.features(g, p, Q, eps, dt)
    params, norm = _params(14), _data_norm(X, 15)
    wq = M.bf16_round(params)
    net = lambda X: M.forward(wq, norm.astype(np.float64), X)
    interior = ~C.boundary_cells(g, p)
    ind0 = np.max(np.abs(net(X)), axis=1).reshape(g.ny, g.nx)
    for thr in _gap_thresholds(ind0, interior):
        Q1, G1, H1, fo, io, ro = C.hybrid_run(g, p, Q, G0, dt, eps, net, thr, nsteps=2)
        if min(np.min(np.abs(i[interior] - thr)) for i in io) / thr > 5e-4:
            break
    stale = fo[1]  # closure cells of the last hybrid step
    none = np.zeros_like(stale)
    Qo, Go, Ho = O.step_closure(g, p, Q1, G1, dt, eps, none, stale, np.zeros((4, g.ny, g.nx)))
    mlp = api.MLP(params, norm)
    with api.Solver(g, p) as s:
        s.set_state(Q, G0)
        s.set_closure(mlp, thr)
        s.set_closure_fallback(0.0, 1)
        s.step(dt, eps, 2)
        s.set_closure(None, 0.0)
        s.step(dt, eps, 1)
        s.sync()
        Qg, Hg = s.get_moments()
        Gg = s.get_g()
    assert np.all(q_rel_err(Qg, Qo) <= 1e-12)
    rho = np.asarray(Q).reshape(6, g.ny, g.nx)[0]
    assert np.max(np.abs(Gg - Go)) <= max(1e-11 * np.max(np.abs(Go)), 64 * ULP * np.max(rho) / eps)
    mlp.close()


def test_hybrid_without_closure_cells_is_the_plain_step_bitwise():
    """A hybrid step in which no cell takes the closure is the plain step bit for bit, from any
    state (three chained single steps) and over consecutive steps (both paths keep the row sums
    of g from which their x sweeps take the moments)."""
    g = I.Grid(nx=17, ny=9, nv1=24, nv2=24)
    p = I.Params(nu=-0.5, bc=(I.SPECULAR, I.SPECULAR, I.PERIODIC, I.PERIODIC))
    Q = I.smooth_state(g, 41)
    G0 = I.seeded_g(g, 42, amp=0.02)
    dt, eps = 1e-3, 1e-2
    mlp = api.MLP(_params(10), _norm(11))

    def run(Q, G, thr, n):
        with api.Solver(g, p) as s:
            s.set_state(Q, G)
            if thr is not None:
                s.set_closure(mlp, thr)  # max |y| <= 0 nowhere: every cell takes the micro path
            s.step(dt, eps, n)
            s.sync()
            Qn, Hn = s.get_moments()
            Gn = s.get_g()
            if thr is not None:
                assert s.closure_stats()[0] == 0
        return Qn, Hn, Gn

    Qc, Gc = Q, G0
    for _ in range(3):
        Qa, Ha, Ga = run(Qc, Gc, None, 1)
        Qb, Hb, Gb = run(Qc, Gc, 0.0, 1)
        assert np.array_equal(Qa, Qb) and np.array_equal(Ha, Hb) and np.array_equal(Ga, Gb)
        Qc, Gc = Qa, Ga
    Qa, Ha, Ga = run(Q, G0, None, 3)
    Qb, Hb, Gb = run(Q, G0, 0.0, 3)
    assert np.array_equal(Qa, Qb) and np.array_equal(Ha, Hb) and np.array_equal(Ga, Gb)
    mlp.close()


def test_closure_rejects_fp32_contexts_and_bad_thresholds():
    g = I.Grid(nx=8, ny=8, nv1=16, nv2=16)
    mlp = api.MLP(_params(12), _norm(13))
    p32 = I.Params(precision=I.PREC_G_FP32)
    with api.Solver(g, p32) as s:
        with pytest.raises(api.MMError):
            s.set_closure(mlp, 1e-3)
    with api.Solver(g, I.Params()) as s:
        for bad in (-1.0, float("nan"), float("inf")):
            with pytest.raises(api.MMError):
                s.set_closure(mlp, bad)
        s.set_closure(None, 0.0)
    mlp.close()


def test_low_closure_fraction_falls_back_to_plain_steps():
    """Below the minimum closure fraction, the steps that follow an evaluation step are plain:
    the first of them the oracle's plain step with the closure cells' g reset to Ghat(Q^n), the
    next ones plain oracle steps; the next evaluation step is hybrid again."""
    g = I.Grid(nx=12, ny=10, nv1=16, nv2=16)
    p = I.Params(nu=-0.5, bc=(I.SPECULAR,) * 4)
    Q = I.smooth_state(g, 51, amp=0.2, umax=0.25, aniso=0.05)
    G0 = I.seeded_g(g, 52, amp=0.02)
    dt, eps = 0.5 / (16.0 * 12 + 16.0 * 10), 1e-2
    X, _, _ = C.features(g, p, Q, eps, dt)
    params, norm = _params(14), _data_norm(X, 15)
    wq = M.bf16_round(params)
    net = lambda X: M.forward(wq, norm.astype(np.float64), X)
    interior = ~C.boundary_cells(g, p)
    ind0 = np.max(np.abs(net(X)), axis=1).reshape(g.ny, g.nx)
    for thr in _gap_thresholds(ind0, interior):
        Q1, G1, H1, fo, io, ro = C.hybrid_run(g, p, Q, G0, dt, eps, net, thr, nsteps=1)
        if min(np.min(np.abs(i[interior] - thr)) for i in io) / thr > 5e-4 and fo[0].sum() > 0:
            break
    none = np.zeros_like(fo[0])
    Q2, G2, H2 = O.step_closure(g, p, Q1, G1, dt, eps, none, fo[0], np.zeros((4, g.ny, g.nx)))
    Qo, Go, Ho = O.step(g, p, Q2, G2, dt, eps, 1)
    mlp = api.MLP(params, norm)
    with api.Solver(g, p) as s:
        s.set_state(Q, G0)
        s.set_closure(mlp, thr)
        s.set_closure_fallback(1.0, 4)  # any closure fraction is below 1: fall back
        s.step(dt, eps, 3)
        s.sync()
        Qg, Hg = s.get_moments()
        Gg = s.get_g()
        assert s.closure_steps() == (1, 2)
        s.step(dt, eps, 2)  # the fourth step is plain, the fifth an evaluation again
        assert s.closure_steps() == (2, 3)
    assert np.all(q_rel_err(Qg, Qo) <= 1e-12)
    rho = np.asarray(Q).reshape(6, g.ny, g.nx)[0]
    assert np.max(np.abs(Gg - Go)) <= max(1e-11 * np.max(np.abs(Go)), 64 * ULP * np.max(rho) / eps)
    mlp.close()
