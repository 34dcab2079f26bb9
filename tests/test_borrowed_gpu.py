"""Contexts on caller-owned device memory (mm_create_borrowed) and the state from primitive fields
(mm_set_state_prim): the borrowed context computes bitwise what an owning context computes, in
the caller's buffers (Q updated in place, g in the caller's buffer after every call, also for FP32
g, which alternates between two buffers inside mm_step), rejects too little scratch and
misaligned buffers; the primitive setter forms exactly the oracle's Q with g = 0."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2509_21832_gb300 import api
from paper_2509_21832_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = [
    ("fp64_specular_32", I.Grid(nx=20, ny=13, nv1=32, nv2=32), I.Params(bc=(I.SPECULAR,) * 4)),
    ("fp64_periodic_16", I.Grid(nx=11, ny=9, nv1=16, nv2=16), I.Params(bc=(I.PERIODIC,) * 4)),
    ("fp32_diffuse_24", I.Grid(nx=14, ny=10, nv1=24, nv2=24),
     I.Params(bc=(I.EXTRAP, I.EXTRAP, I.DIFFUSE, I.EXTRAP), precision=I.PREC_G_FP32)),
]


def borrow_tensors(grid, params):
    nc = grid.nx * grid.ny
    gdt = torch.float32 if params.precision == I.PREC_G_FP32 else torch.float64
    Q = torch.empty(6 * nc, dtype=torch.float64, device="cuda")
    G = torch.empty(nc * grid.nv1 * grid.nv2, dtype=gdt, device="cuda")
    S = torch.empty(api.mm_scratch_bytes(grid, params), dtype=torch.uint8, device="cuda")
    return Q, G, S


@pytest.mark.parametrize("name,grid,params", CASES, ids=[c[0] for c in CASES])
def test_borrowed_context_matches_owned(name, grid, params):
    Q0 = I.smooth_state(grid, seed=3, umax=0.2, aniso=0.05)
    G0 = I.seeded_g(grid, seed=4, amp=0.02)
    dt = 0.4 / (8.0 * grid.nx + 8.0 * grid.ny)
    eps = 1e-2
    with api.Solver(grid, params) as s:
        s.set_state(Q0, G0)
        s.step(dt, eps, 3)  # an odd count: FP32 g ends in the other buffer of its pair
        Qa, Ha = s.get_moments()
        Ga = s.get_g()
    Qt, Gt, St = borrow_tensors(grid, params)
    with api.Solver(grid, params, borrow=(Qt, Gt, St)) as b:
        b.set_state(Q0, G0)
        b.step(dt, eps, 3)
        Qb, Hb = b.get_moments()
        Gb = b.get_g()
        torch.cuda.synchronize()
        assert np.array_equal(Qa, Qb) and np.array_equal(Ha, Hb) and np.array_equal(Ga, Gb), name
        # the state is in the caller's tensors
        assert np.array_equal(Qt.cpu().numpy().reshape(Qa.shape), Qa), name
        assert np.array_equal(Gt.double().cpu().numpy().reshape(Ga.shape), Ga), name
        b.step(dt, eps, 2)
        Qc, _ = b.get_moments()
        torch.cuda.synchronize()
        assert np.array_equal(Qt.cpu().numpy().reshape(Qc.shape), Qc), name
    # the caller's tensors outlive the context and keep the last state
    assert np.array_equal(Qt.cpu().numpy().reshape(Qc.shape), Qc)


def test_borrowed_context_rejects_bad_buffers():
    grid, params = CASES[0][1], CASES[0][2]
    Qt, Gt, St = borrow_tensors(grid, params)
    with pytest.raises(api.MMError) as e:
        api.Solver(grid, params, borrow=(Qt, Gt, St[:-1]))
    assert e.value.status == api.MM_ERR_INVALID_ARG
    Gx = torch.empty(Gt.numel() + 1, dtype=Gt.dtype, device="cuda")[1:]  # 8 bytes off
    with pytest.raises(api.MMError) as e:
        api.Solver(grid, params, borrow=(Qt, Gx, St))
    assert e.value.status == api.MM_ERR_INVALID_ARG


@pytest.mark.parametrize("prec", [I.PREC_FP64, I.PREC_G_FP32])
def test_set_state_prim_matches_oracle(prec):
    grid = I.Grid(nx=17, ny=11, nv1=24, nv2=24)
    params = I.Params(bc=(I.PERIODIC,) * 4, precision=prec)
    rng = np.random.default_rng(11)
    shape = (grid.ny, grid.nx)
    rho = rng.uniform(0.2, 2.0, shape)
    u1, u2 = rng.uniform(-0.6, 0.6, shape), rng.uniform(-0.6, 0.6, shape)
    T = rng.uniform(0.5, 2.0, shape)
    Qo = O.q_from_prim(rho, u1, u2, T)
    dt = 0.4 / (8.0 * grid.nx + 8.0 * grid.ny)
    with api.Solver(grid, params) as s:
        s.set_state_prim(rho, u1, u2, T)
        Q, _ = s.get_moments()
        assert np.array_equal(Q, Qo)
        assert not np.any(s.get_g())
        s.step(dt, 1e-2, 2)
        Q2, H2 = s.get_moments()
        # a rejected field leaves the state as it was
        bad = T.copy()
        bad[3, 4] = 0.0
        with pytest.raises(api.MMError) as e:
            s.set_state_prim(rho, u1, u2, bad)
        assert e.value.status == api.MM_ERR_INVALID_ARG
        Q3, _ = s.get_moments()
        assert np.array_equal(Q3, Q2)
    with api.Solver(grid, params) as s:
        s.set_state(Qo, None)
        s.step(dt, 1e-2, 2)
        Q4, H4 = s.get_moments()
    assert np.array_equal(Q2, Q4) and np.array_equal(H2, H4)
