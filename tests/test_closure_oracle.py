"""Pins of the closure oracle (network, features, Chapman-Enskog heat flux, hybrid step) to
facts fixed by mathematics: BF16 rounding by enumeration, the normal CDF, finite differences of
the loss, closed-form gradients, the first Adam step, moments of the oracle's own Ghat by
quadrature, invariances of the features, and conservation of the hybrid step."""
import math

import numpy as np

from oracle import closure_oracle as C
from oracle import mlp_oracle as M
from oracle import oracle as O
from paper_2509_21832_gb300 import inputs as I


# ---------------------------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------------------------
def test_bf16_rounding_by_enumeration():
    # ties go to the even mantissa
    assert M.bf16_round(np.float32(1.0 + 2.0 ** -8))[()] == 1.0
    assert M.bf16_round(np.float32(1.0 + 3 * 2.0 ** -8))[()] == 1.0 + 2.0 ** -6
    assert M.bf16_round(np.float32(1.0 + 2.0 ** -8 + 2.0 ** -20))[()] == 1.0 + 2.0 ** -7
    assert M.bf16_round(np.float32(-3.0))[()] == -3.0
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(2000) * np.exp(rng.uniform(-20, 20, 2000))).astype(np.float32)
    r = M.bf16_round(x)
    for xi, ri in zip(x.astype(np.float64), r):
        # the two BF16 neighbours of x: truncation and truncation + one ulp (same sign)
        e = math.floor(math.log2(abs(xi)))
        ulp = 2.0 ** (e - 7)
        lo = math.floor(abs(xi) / ulp) * ulp
        cands = [lo, lo + ulp]
        best = min(cands, key=lambda c: (abs(c - abs(xi)), (round(c / ulp) % 2)))
        assert abs(ri) == best and (ri == 0 or math.copysign(1, ri) == math.copysign(1, xi))


def test_gelu_is_z_times_normal_cdf():
    assert M.gelu(np.array(0.0)) == 0.0
    # Phi(1) = 0.841344746068543 (normal distribution tables)
    assert abs(M.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    assert abs(M.gelu(np.array(-1.0)) + (1 - 0.8413447460685429)) < 1e-15
    assert abs(M.gelu(np.array(8.0)) - 8.0) < 1e-13 and abs(M.gelu(np.array(-8.0))) < 1e-13
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - M.gelu_grad(z))) < 1e-8


def _data(seed, n=40):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, M.N_IN)) * 0.7 + 0.1
    T = rng.standard_normal((n, M.N_OUT))
    norm = np.concatenate([rng.standard_normal(M.N_IN) * 0.1, np.exp(rng.uniform(-0.3, 0.3, M.N_IN)),
                           rng.standard_normal(M.N_OUT) * 0.1, np.exp(rng.uniform(-0.3, 0.3, M.N_OUT))])
    return X, T, norm


def test_gradient_matches_central_differences():
    X, T, norm = _data(1)
    p = M.init_params(3).astype(np.float64)
    p[M.OFF_B1:M.OFF_W2] = 0.05
    p[M.OFF_B3:] = 0.1
    L, g = M.loss_and_grad(p, norm, X, T)
    assert abs(L - M.loss(p, norm, X, T)) < 1e-14 * max(1.0, L)
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.choice(M.N_PARAM, 60, replace=False),
                          [M.OFF_B1, M.OFF_W2 + 7, M.OFF_B2 + 3, M.OFF_W3 + 5, M.OFF_B3 + 2]])
    h = 1e-5
    for q in idx:
        pp, pm = p.copy(), p.copy()
        pp[q] += h
        pm[q] -= h
        fd = (M.loss(pp, norm, X, T) - M.loss(pm, norm, X, T)) / (2 * h)
        assert abs(fd - g[q]) <= 1e-7 * max(1.0, np.max(np.abs(g))), q


def test_gradient_closed_form_with_zero_output_layer():
    # W3 = 0: y' = b3 for every sample, so dL/db3 = (2/n) sum_s (b3 - t'_s) and all other
    # gradients vanish
    X, T, norm = _data(4)
    p = M.init_params(5).astype(np.float64)
    p[M.OFF_W3:M.OFF_B3] = 0.0
    p[M.OFF_B3:] = [0.3, -0.2, 0.1, 0.05]
    L, g = M.loss_and_grad(p, norm, X, T)
    ts = (T - norm[2 * M.N_IN:2 * M.N_IN + M.N_OUT]) / norm[2 * M.N_IN + M.N_OUT:]
    b3 = p[M.OFF_B3:]
    assert abs(L - np.sum((b3 - ts) ** 2) / len(X)) < 1e-13
    assert np.allclose(g[M.OFF_B3:], 2.0 * np.sum(b3 - ts, axis=0) / len(X), atol=1e-14, rtol=0)
    assert np.all(g[:M.OFF_W3] == 0.0)
    # and dL/dW3[o][i] = (2/n) sum_s (b3_o - t'_so) a2_si, a2 from the hidden layers
    a2 = M._forward(p, norm, X)[4]
    assert np.allclose(g[M.OFF_W3:M.OFF_B3].reshape(M.N_OUT, M.N_HIDDEN),
                       (2.0 / len(X)) * (b3 - ts).T @ a2, atol=1e-13, rtol=0)


def test_bf16_operand_gradient_reduces_to_the_chain_rule_and_stays_close():
    """The training kernels' gradient with BF16 operands: with the rounding replaced by the
    identity it is the plain chain-rule gradient (itself pinned by central differences above);
    with BF16 rounding of the activations and back-propagated gradients it stays within a few
    BF16 units (2^-8 relative) of it in every layer, and differs from it (the roundings act)."""
    X, T, norm = _data(1)
    p = M.bf16_round(M.init_params(3))
    L0, g0 = M.loss_and_grad(p, norm, X, T)
    Li, gi = M.loss_and_grad_bf16(p, norm, X, T, rnd=lambda a: a)
    assert abs(Li - L0) <= 1e-14 * max(1.0, L0)
    assert np.max(np.abs(gi - g0)) <= 1e-14 * np.max(np.abs(g0))
    Lb, gb = M.loss_and_grad_bf16(p, norm, X, T)
    assert abs(Lb - L0) <= 2.0 ** -6 * L0
    for a, b in ((M.OFF_W1, M.OFF_B1), (M.OFF_W2, M.OFF_B2), (M.OFF_W3, M.OFF_B3)):
        scale = np.max(np.abs(g0[a:b]))
        err = np.max(np.abs(gb[a:b] - g0[a:b]))
        assert 0.0 < err <= 2.0 ** -5 * scale, (a, err / scale)


def test_first_adam_step_moves_by_lr_times_sign():
    g = np.array([3.0, -1e-3, 0.5, -7.0])
    w, m1, m2 = M.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, 1e-2)
    assert np.allclose(w, -1e-2 * np.sign(g), rtol=1e-4, atol=0)
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)


# ---------------------------------------------------------------------------------------------
# features and the Chapman-Enskog heat flux
# ---------------------------------------------------------------------------------------------
def _smooth_case(n=10, nv=40, vmax=12.0, seed=3, bc=(I.PERIODIC,) * 4, tau_model=I.TAU_RHO):
    g = I.Grid(nx=n, ny=n, nv1=nv, nv2=nv, v1min=-vmax, v1max=vmax, v2min=-vmax, v2max=vmax)
    p = I.Params(nu=-0.5, bc=bc, tau_model=tau_model)
    Q = I.smooth_state(g, seed, amp=0.2, umax=0.3, aniso=0.0)
    return g, p, Q


def test_h_ce_equals_moments_of_ghat():
    # eps dv^2 sum c (x) c (x) c Ghat over a wide velocity box reproduces the closed form
    for eps in (1e-2, 1e-1):
        g, p, Q = _smooth_case()
        X, Hce, scale = C.features(g, p, Q, eps, 1e-3)
        Gh = O.ghat(g, p, Q, eps).reshape(g.ny, g.nx, g.nv2, g.nv1)
        v1, v2 = g.v1(), g.v2()
        dv = (g.v1max - g.v1min) / g.nv1 * (g.v2max - g.v2min) / g.nv2
        Qr = Q.reshape(6, g.ny, g.nx)
        u1, u2 = Qr[1] / Qr[0], Qr[2] / Qr[0]
        c1 = v1[None, None, None, :] - u1[:, :, None, None]
        c2 = v2[None, None, :, None] - u2[:, :, None, None]
        Hq = np.stack([np.sum(c1 ** 3 * Gh, axis=(2, 3)), np.sum(c1 ** 2 * c2 * Gh, axis=(2, 3)),
                       np.sum(c1 * c2 ** 2 * Gh, axis=(2, 3)), np.sum(c2 ** 3 * Gh, axis=(2, 3))])
        Hq *= eps * dv
        assert np.max(np.abs(Hq - Hce)) <= 1e-9 * np.max(np.abs(Hce)), eps


def test_features_of_a_uniform_state():
    g = I.Grid(nx=5, ny=4, nv1=8, nv2=8)
    p = I.Params(nu=-0.5, bc=(I.SPECULAR, I.EXTRAP, I.PERIODIC, I.PERIODIC))
    rho, U1, U2, T = 1.7, 0.3, -0.2, 1.3
    Q = I.q_from_prims(np.full((4, 5), rho), np.full((4, 5), U1), np.full((4, 5), U2),
                       np.full((4, 5), T))
    eps, dt = 3e-2, 1e-3
    X, Hce, scale = C.features(g, p, Q, eps, dt)
    inner = X.reshape(4, 5, 39)[:, 1:]  # away from the specular wall the neighbours agree
    assert np.all(inner[..., :32] == 0.0)
    assert np.allclose(X[:, 34], U1 / math.sqrt(T), rtol=1e-15, atol=0)
    assert np.allclose(X[:, 35], U2 / math.sqrt(T), rtol=1e-15, atol=0)
    assert np.all(X[:, 36] == math.log10(eps))
    assert np.allclose(X[:, 37], eps / (eps + dt * rho), rtol=1e-15)  # tau = rho
    k = eps * math.sqrt(T) / (rho * 0.2)  # h = min(1/5, 1/4)
    assert np.allclose(X[:, 38], math.log10(k), rtol=0, atol=1e-15)
    assert np.all(Hce == 0.0)
    assert np.allclose(scale, eps * rho * T ** 1.5, rtol=1e-15)
    # at the specular wall the mirror image has u1 -> -u1: the left neighbours see -2 U1
    wall = X.reshape(4, 5, 39)[:, 0]
    for nb in (0, 3, 5):  # (di = -1) in rows j-1, j, j+1
        assert np.allclose(wall[:, 4 * nb + 1], -2 * k * U1 / math.sqrt(T), rtol=1e-14)


def test_features_translation_boost_and_scaling():
    g, p, Q = _smooth_case(n=8, nv=8, tau_model=I.TAU_CONST)
    eps, dt = 1e-2, 2e-3
    X, Hce, s = C.features(g, p, Q, eps, dt)
    # periodic translation by one cell in each direction
    Qs = np.roll(np.roll(Q.reshape(6, 8, 8), 1, axis=1), 2, axis=2)
    Xs, Hs, ss = C.features(g, p, Qs, eps, dt)
    assert np.allclose(Xs.reshape(8, 8, 39), np.roll(np.roll(X.reshape(8, 8, 39), 1, 0), 2, 1),
                       rtol=0, atol=1e-14)
    # Galilean boost: only features 34, 35 change (by U / sqrt T); H_CE unchanged
    Qr = Q.reshape(6, 8, 8)
    rho, u1, u2 = Qr[0], Qr[1] / Qr[0], Qr[2] / Qr[0]
    P11 = Qr[3] - rho * u1 ** 2
    P12 = Qr[4] - rho * u1 * u2
    P22 = Qr[5] - rho * u2 ** 2
    U = (0.4, -0.25)
    w1, w2 = u1 + U[0], u2 + U[1]
    Qb = np.stack([rho, rho * w1, rho * w2, P11 + rho * w1 ** 2, P12 + rho * w1 * w2, P22 + rho * w2 ** 2])
    Xb, Hb, sb = C.features(g, p, Qb, eps, dt)
    assert np.allclose(Xb[:, :34], X[:, :34], rtol=0, atol=1e-12)
    assert np.allclose(Xb[:, 36:], X[:, 36:], rtol=0, atol=1e-15)
    T = (P11 + P22) / (2 * rho)
    assert np.allclose(Xb[:, 34] - X[:, 34], (U[0] / np.sqrt(T)).ravel(), atol=1e-12)
    assert np.allclose(Hb, Hce, rtol=0, atol=1e-12 * np.max(np.abs(Hce)))
    # rho -> 2 rho at constant tau: features 0..35 unchanged, H_CE and the scale double
    Xd, Hd, sd = C.features(g, p, 2.0 * Q, eps, dt)
    assert np.allclose(Xd, X, rtol=0, atol=1e-13)
    assert np.allclose(Hd, 2.0 * Hce, rtol=1e-13, atol=0) and np.allclose(sd, 2.0 * s, rtol=1e-14)


def test_stencil_features_are_resolution_independent():
    # a smooth field on an n and a 3n grid: cell i of the coarse grid and cell 3i+1 of the fine
    # grid share a centre; the Knudsen-scaled neighbour differences agree to O(h) (about 4.4 h
    # relative for the diagonal density differences of this field, from the second-order terms
    # of the Taylor expansion), while a missing 1/h would put them a factor 3 apart
    def q_on(n):
        g = I.Grid(nx=n, ny=n, nv1=8, nv2=8)
        x, y = np.meshgrid(g.xc(), g.yc())
        rho = 1.0 + 0.3 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
        T = 1.0 + 0.2 * np.cos(2 * np.pi * (x + y))
        u1 = 0.2 * np.sin(2 * np.pi * y)
        u2 = 0.1 * np.cos(2 * np.pi * x)
        return g, I.q_from_prims(rho, u1, u2, T)
    p = I.Params(nu=-0.5, bc=(I.PERIODIC,) * 4)
    gc, Qc = q_on(32)
    gf, Qf = q_on(96)
    Xc = C.features(gc, p, Qc, 1e-2, 1e-3)[0].reshape(32, 32, 39)
    Xf = C.features(gf, p, Qf, 1e-2, 1e-3)[0].reshape(96, 96, 39)[1::3, 1::3]
    d = np.max(np.abs(Xf[..., :32] - Xc[..., :32]))
    assert d <= 0.2 * np.max(np.abs(Xc[..., :32])), d
    # log10 k moves by log10 3 between the grids
    assert np.allclose(Xf[..., 38] - Xc[..., 38], np.log10(3.0), atol=1e-12)


# ---------------------------------------------------------------------------------------------
# hybrid step
# ---------------------------------------------------------------------------------------------
def test_closure_step_without_closure_cells_is_the_plain_step():
    g, p, Q = _smooth_case(n=6, nv=8)
    G0 = I.seeded_g(g, 4, amp=0.02)
    none = np.zeros((g.ny, g.nx), dtype=bool)
    Hcl = np.full((4, g.ny, g.nx), 123.0)
    a = O.step(g, p, Q, G0, 1e-3, 1e-2)
    b = O.step_closure(g, p, Q, G0, 1e-3, 1e-2, none, none, Hcl)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    # refreshing every cell is the plain step from g^n = Ghat(Q^n)
    alls = np.ones((g.ny, g.nx), dtype=bool)
    a = O.step(g, p, Q, O.ghat(g, p, Q, 1e-2), 1e-3, 1e-2)
    b = O.step_closure(g, p, Q, G0, 1e-3, 1e-2, none, alls, Hcl)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_closure_cells_keep_g_take_the_given_heat_flux_and_conserve():
    g, p, Q = _smooth_case(n=8, nv=12)
    G0 = I.seeded_g(g, 5, amp=0.02)
    eps, dt = 1e-2, 1e-3
    flags = np.zeros((g.ny, g.nx), dtype=bool)
    flags[2:6, 3:7] = True
    refresh = C.needed_cells(g, p, ~flags) & flags  # the closure ring
    rng = np.random.default_rng(0)
    Hcl = rng.standard_normal((4, g.ny, g.nx)) * 1e-3
    Qn, Gn, Hn = O.step_closure(g, p, Q, G0, dt, eps, flags, refresh, Hcl)
    Gh = O.ghat(g, p, Q, eps).reshape(g.ny, g.nx, -1)
    Gn = Gn.reshape(g.ny, g.nx, -1)
    G0r = G0.reshape(g.ny, g.nx, -1)
    assert np.array_equal(Gn[refresh], Gh[refresh])
    assert np.array_equal(Gn[flags & ~refresh], G0r[flags & ~refresh])
    assert np.array_equal(Hn[:, flags], Hcl[:, flags])
    # the ring is one cell wide around the micro cells (3x3 blocks)
    assert refresh.sum() == 12 and not refresh[3:5, 4:6].any()
    # micro cells far from the refreshed ring keep the plain step's micro solution
    Qp, Gp, Hp = O.step(g, p, Q, G0, dt, eps)
    far = ~C.needed_cells(g, p, refresh) & ~flags
    assert far.sum() > 0
    assert np.array_equal(Gn[far], Gp.reshape(g.ny, g.nx, -1)[far])
    assert np.array_equal(Hn[:, far], Hp[:, far])
    # the heat flux enters the macro update in conservation form: totals are kept
    tot0 = Q.reshape(6, -1).sum(axis=1)
    tot1 = Qn.reshape(6, -1).sum(axis=1)
    for m in (0, 1, 2):
        assert abs(tot1[m] - tot0[m]) <= 1e-12 * max(1.0, abs(tot0[m]))
    assert abs((tot1[3] + tot1[5]) - (tot0[3] + tot0[5])) <= 1e-12 * abs(tot0[3] + tot0[5])


def test_needed_cells_are_the_3x3_blocks_with_boundary_rules():
    g = I.Grid(nx=7, ny=5)
    m = np.zeros((5, 7), dtype=bool)
    m[0, 0] = True
    per = I.Params(bc=(I.PERIODIC,) * 4)
    wall = I.Params(bc=(I.SPECULAR,) * 4)
    a = C.needed_cells(g, per, m)
    b = C.needed_cells(g, wall, m)
    assert a.sum() == 9 and a[4, 6] and a[1, 1] and a[4, 0] and a[0, 6]
    assert b.sum() == 4 and b[1, 1] and not b[4, 6]
