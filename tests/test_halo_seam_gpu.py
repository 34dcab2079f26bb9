"""The spatial block decomposition through the library on one GPU: 2 x 2 (and 3 x 2) blocks,
each a context working in its own CUDA tensors (mm_create_borrowed), halos of two cells refreshed
by device-local copies before every step (the seam that a multi-GPU run would exchange between
devices), reproduce the undivided step bit for bit: Q and g of every owned cell after several
steps, for the one-row-per-pass meshes with row sums (32^2) and the two-row meshes (16^2), with
periodic, specular and diffuse domain sides."""
import numpy as np
import pytest
import torch

from paper_2509_21832_gb300 import api, halo
from paper_2509_21832_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = [
    ("periodic_32", 32, (I.PERIODIC,) * 4, 2, 2, I.PREC_FP64),
    ("specular_diffuse_16", 16, (I.PERIODIC, I.PERIODIC, I.SPECULAR, I.DIFFUSE), 3, 2, I.PREC_FP64),
    ("extrap_specular_32", 32, (I.EXTRAP, I.SPECULAR, I.PERIODIC, I.PERIODIC), 2, 2, I.PREC_FP64),
    ("fp32_g_specular_diffuse_24", 24, (I.PERIODIC, I.PERIODIC, I.DIFFUSE, I.SPECULAR), 2, 2,
     I.PREC_G_FP32),
]


@pytest.mark.parametrize("name,nv,bc,px,py,prec", CASES, ids=[c[0] for c in CASES])
def test_blocks_on_one_gpu_reproduce_the_undivided_step(name, nv, bc, px, py, prec):
    grid = I.Grid(nx=24, ny=16, x0=0.0, x1=1.5, y0=0.0, y1=1.0, nv1=nv, nv2=nv)
    params = I.Params(bc=bc, precision=prec)
    Q = I.smooth_state(grid, seed=31, umax=0.25, aniso=0.06)
    G = I.seeded_g(grid, seed=32, amp=0.02)
    dt = 0.4 / (8.0 * grid.nx + 8.0 * grid.ny)
    eps, steps = 1e-2, 4
    with api.Solver(grid, params) as s:
        s.set_state(Q, G)
        s.step(dt, eps, steps)
        Qu, _ = s.get_moments()
        Gu = s.get_g()
    blocks = halo.decompose(grid, params, px, py, w=2)
    copies = halo.plan(blocks)
    gdt = torch.float32 if prec == I.PREC_G_FP32 else torch.float64
    Gsrc = torch.from_numpy(G).to(gdt)
    states = [(Qb.cuda(), Gb.cuda()) for Qb, Gb in
              halo.scatter(blocks, torch.from_numpy(Q), Gsrc)]
    solvers = []
    for b, (Qb, Gb) in zip(blocks, states):
        S = torch.empty(api.mm_scratch_bytes(b.grid, b.params), dtype=torch.uint8, device="cuda")
        sv = api.Solver(b.grid, b.params, borrow=(Qb, Gb, S))
        sv.scratch = S
        solvers.append(sv)
    try:
        for n in range(steps):
            if n:
                halo.exchange_local(blocks, copies, states)
            for sv, (Qb, Gb) in zip(solvers, states):
                # halos in (row sums re-formed); FP32 g goes in through its FP64 image, which
                # rounds back to the same FP32 values
                sv.set_state(Qb.clone(), Gb.double())
                sv.step(dt, eps, 1)
        for sv in solvers:
            sv.sync()
        Qs, Gs = torch.zeros(Q.shape, dtype=torch.float64), torch.zeros(G.shape, dtype=torch.float64)
        halo.gather(blocks, [(Qb.cpu(), Gb.cpu().double()) for Qb, Gb in states], Qs, Gs)
    finally:
        for sv in solvers:
            sv.close()
    assert np.array_equal(Qs.numpy(), Qu), name
    assert np.array_equal(Gs.numpy(), Gu), name


@pytest.mark.parametrize("name,nv,bc,px,py,prec", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_blocks_with_region_refresh_reproduce_the_undivided_step(name, nv, bc, px, py, prec):
    """The same with the halo refresh that `bench.py --decompose` uses: after the exchange only
    the halo rectangles' g is re-registered (mm_g_region_changed re-forms their row sums); the
    state is set once."""
    grid = I.Grid(nx=24, ny=16, x0=0.0, x1=1.5, y0=0.0, y1=1.0, nv1=nv, nv2=nv)
    params = I.Params(bc=bc, precision=prec)
    Q = I.smooth_state(grid, seed=41, umax=0.25, aniso=0.06)
    G = I.seeded_g(grid, seed=42, amp=0.02)
    dt = 0.4 / (8.0 * grid.nx + 8.0 * grid.ny)
    eps, steps = 1e-2, 4
    with api.Solver(grid, params) as s:
        s.set_state(Q, G)
        s.step(dt, eps, steps)
        Qu, _ = s.get_moments()
        Gu = s.get_g()
    blocks = halo.decompose(grid, params, px, py, w=2)
    copies = halo.plan(blocks)
    states = [(Qb.cuda(), Gb.cuda()) for Qb, Gb in
              halo.scatter(blocks, torch.from_numpy(Q), torch.from_numpy(G))]
    solvers = []
    for b, (Qb, Gb) in zip(blocks, states):
        S = torch.empty(api.mm_scratch_bytes(b.grid, b.params), dtype=torch.uint8, device="cuda")
        sv = api.Solver(b.grid, b.params, stream=torch.cuda.current_stream().cuda_stream,
                        borrow=(Qb, Gb, S))
        sv.scratch = S
        sv.set_state(Qb.clone(), Gb.clone())
        solvers.append(sv)
    try:
        for n in range(steps):
            if n:
                halo.exchange_local(blocks, copies, states)
                for b, sv in zip(blocks, solvers):
                    for r in halo.halo_regions(b):
                        sv.g_region_changed(*r)
            for sv in solvers:
                sv.step(dt, eps, 1)
        for sv in solvers:
            sv.sync()
        Qs, Gs = torch.zeros(Q.shape, dtype=torch.float64), torch.zeros(G.shape, dtype=torch.float64)
        halo.gather(blocks, [(Qb.cpu(), Gb.cpu()) for Qb, Gb in states], Qs, Gs)
    finally:
        for sv in solvers:
            sv.close()
    assert np.array_equal(Qs.numpy(), Qu), name
    assert np.array_equal(Gs.numpy(), Gu), name
    with pytest.raises(api.MMError):
        solvers_bad = api.Solver(grid, params)
        try:
            solvers_bad.set_state(Q, G)
            solvers_bad.g_region_changed(0, grid.nx + 1, 0, 1)
        finally:
            solvers_bad.close()


def test_decomposed_bench_stepper_on_one_block():
    """The GPU stepper of `bench.py --decompose` (a borrowed context on the block's tensors) on a
    single rank, where the one block is the whole grid: the same state as a plain context after
    the same steps, bit for bit."""
    import bench
    pr = I.bump_specular(n=48, nv=32, eps=1e-2, seed=4)
    b, Qt, Gt, sec = bench.run_blocks(pr, 1, 0, 3, 0, bench.gpu_block_stepper,
                                      torch.device("cuda"))
    torch.cuda.synchronize()
    with api.Solver(pr.grid, pr.params) as s:
        s.set_state(pr.Q, pr.G)
        s.step(pr.dt, pr.eps, 3)
        Qu, _ = s.get_moments()
        Gu = s.get_g()
    assert sec > 0
    assert np.array_equal(Qt.cpu().numpy().reshape(Qu.shape), Qu)
    assert np.array_equal(Gt.cpu().numpy().reshape(Gu.shape), Gu)
