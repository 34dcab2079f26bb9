"""The spatial block decomposition (paper_2509_21832_gb300/halo.py) on CPU: blocks with halos of
two cells, refreshed before every step, reproduce the undivided step bit for bit.  The blocks are
stepped by the oracle (the library needs a GPU; tests/test_halo_seam_gpu.py runs the same
decomposition through it), in one process (local copies) and as two gloo ranks that exchange
their face cells point to point."""
import os
import socket
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_21832_gb300 import halo
from paper_2509_21832_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS = 3


def problem(bc):
    grid = I.Grid(nx=16, ny=12, x0=0.0, x1=1.0, y0=0.0, y1=0.75, nv1=8, nv2=8)
    params = I.Params(bc=bc)
    Q = I.smooth_state(grid, seed=21, umax=0.25, aniso=0.06)
    G = I.seeded_g(grid, seed=22, amp=0.02)
    dt = 0.4 / (8.0 * grid.nx + 8.0 * grid.ny)
    return grid, params, Q, G, dt, 1e-2


def test_decompose_geometry():
    grid, params, *_ = problem((I.PERIODIC, I.PERIODIC, I.SPECULAR, I.SPECULAR))
    blocks = halo.decompose(grid, params, 3, 2, w=2)
    owned = np.zeros(grid.nx * grid.ny, dtype=int)
    for b in blocks:
        g = b.global_index()[b.owned_mask()]
        owned[g] += 1
        # cell sizes bitwise those of the undivided grid
        assert (b.grid.x1 - b.grid.x0) / b.grid.nx == (grid.x1 - grid.x0) / grid.nx
        assert (b.grid.y1 - b.grid.y0) / b.grid.ny == (grid.y1 - grid.y0) / grid.ny
        # x is periodic: halos on both x sides; y keeps the specular walls of the domain
        assert b.hl == b.hr == 2
        assert b.hb == (0 if b.by == 0 else 2) and b.ht == (0 if b.by == 1 else 2)
        assert b.params.bc[2] == (I.SPECULAR if b.by == 0 else I.EXTRAP)
    assert np.all(owned == 1)  # every cell owned exactly once
    copies = halo.plan(blocks)
    for b in blocks:  # every halo cell is refreshed exactly once
        got = np.zeros(b.nx * b.ny, dtype=int)
        for (s, r), (src, dst) in copies.items():
            if r == b.rank:
                got[dst] += 1
                assert np.array_equal(blocks[s].global_index()[src], b.global_index()[dst])
        assert np.array_equal(got, (~b.owned_mask()).astype(int))
    with pytest.raises(ValueError):
        halo.decompose(grid, params, 2, 2, w=1)


@pytest.mark.parametrize("bc,px,py", [
    ((I.PERIODIC,) * 4, 2, 2),
    ((I.PERIODIC, I.PERIODIC, I.SPECULAR, I.DIFFUSE), 2, 3),
    ((I.EXTRAP, I.SPECULAR, I.PERIODIC, I.PERIODIC), 3, 1),
])
def test_blocks_reproduce_the_undivided_step(bc, px, py):
    grid, params, Q, G, dt, eps = problem(bc)
    Qu, Gu, Hu = O.step(grid, params, Q, G, dt, eps, STEPS)
    blocks = halo.decompose(grid, params, px, py, w=2)
    copies = halo.plan(blocks)
    states = halo.scatter(blocks, Q, G)
    for n in range(STEPS):
        if n:
            halo.exchange_local(blocks, copies, states)
        states = [O.step(b.grid, b.params, Qb, Gb, dt, eps, 1)[:2]
                  for b, (Qb, Gb) in zip(blocks, states)]
    Qs, Gs = np.zeros_like(Q), np.zeros_like(G)
    halo.gather(blocks, states, Qs, Gs)
    assert np.array_equal(Qs, Qu) and np.array_equal(Gs, Gu)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import oracle as Orc
    from paper_2509_21832_gb300 import halo as hl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    grid, params, Q, G, dt, eps = problem((I.PERIODIC, I.PERIODIC, I.SPECULAR, I.SPECULAR))
    blocks = hl.decompose(grid, params, world, 1, w=2)
    copies = hl.plan(blocks)
    Qb, Gb = hl.scatter(blocks, Q, G)[rank]
    b = blocks[rank]
    for n in range(STEPS):
        if n:
            Qt, Gt = torch.from_numpy(Qb), torch.from_numpy(Gb)
            hl.exchange(blocks, copies, rank, Qt, Gt)
        Qb, Gb, _ = Orc.step(b.grid, b.params, Qb, Gb, dt, eps, 1)
    dist.barrier()
    out.put((rank, Qb, Gb))
    dist.destroy_process_group()


def test_two_gloo_ranks_exchange_faces_point_to_point():
    import torch.multiprocessing as mp
    grid, params, Q, G, dt, eps = problem((I.PERIODIC, I.PERIODIC, I.SPECULAR, I.SPECULAR))
    Qu, Gu, _ = O.step(grid, params, Q, G, dt, eps, STEPS)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(2)), key=lambda t: t[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    blocks = halo.decompose(grid, params, 2, 1, w=2)
    Qs, Gs = np.zeros_like(Q), np.zeros_like(G)
    halo.gather(blocks, [(Qb, Gb) for _, Qb, Gb in res], Qs, Gs)
    assert np.array_equal(Qs, Qu) and np.array_equal(Gs, Gu)


def test_stale_halos_change_the_result():
    """Without the refresh the blocks diverge from the undivided step (the exchange above is
    what makes them agree)."""
    grid, params, Q, G, dt, eps = problem((I.PERIODIC,) * 4)
    Qu, Gu, _ = O.step(grid, params, Q, G, dt, eps, STEPS)
    blocks = halo.decompose(grid, params, 2, 2, w=2)
    states = halo.scatter(blocks, Q, G)
    for n in range(STEPS):
        states = [O.step(b.grid, b.params, Qb, Gb, dt, eps, 1)[:2]
                  for b, (Qb, Gb) in zip(blocks, states)]
    Qs, Gs = np.zeros_like(Q), np.zeros_like(G)
    halo.gather(blocks, states, Qs, Gs)
    assert not np.array_equal(Qs, Qu) and not np.array_equal(Gs, Gu)


@pytest.mark.parametrize("nx,ny,px,py,w", [(17, 13, 3, 2, 2), (16, 12, 2, 2, 3), (15, 9, 4, 1, 2)])
def test_uneven_blocks_and_wider_halos(nx, ny, px, py, w):
    """Block sizes that do not divide the grid (owned widths differ by one) and a halo wider than
    needed give the undivided step as well; the extended grids keep the undivided cell sizes."""
    grid = I.Grid(nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=0.8, nv1=8, nv2=8)
    params = I.Params(bc=(I.PERIODIC, I.PERIODIC, I.SPECULAR, I.EXTRAP))
    Q = I.smooth_state(grid, seed=41, umax=0.25, aniso=0.06)
    G = I.seeded_g(grid, seed=42, amp=0.02)
    dt = 0.4 / (8.0 * grid.nx + 8.0 * grid.ny)
    Qu, Gu, _ = O.step(grid, params, Q, G, dt, 1e-2, STEPS)
    blocks = halo.decompose(grid, params, px, py, w=w)
    for b in blocks:
        assert (b.grid.x1 - b.grid.x0) / b.grid.nx == (grid.x1 - grid.x0) / grid.nx
        assert (b.grid.y1 - b.grid.y0) / b.grid.ny == (grid.y1 - grid.y0) / grid.ny
    copies = halo.plan(blocks)
    states = halo.scatter(blocks, Q, G)
    for n in range(STEPS):
        if n:
            halo.exchange_local(blocks, copies, states)
        states = [O.step(b.grid, b.params, Qb, Gb, dt, 1e-2, 1)[:2]
                  for b, (Qb, Gb) in zip(blocks, states)]
    Qs, Gs = np.zeros_like(Q), np.zeros_like(G)
    halo.gather(blocks, states, Qs, Gs)
    assert np.array_equal(Qs, Qu) and np.array_equal(Gs, Gu)


def _rank2d(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import oracle as Orc
    from paper_2509_21832_gb300 import halo as hl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    grid, params, Q, G, dt, eps = problem((I.PERIODIC,) * 4)
    blocks = hl.decompose(grid, params, 2, 2, w=2)
    copies = hl.plan(blocks)
    Qb, Gb = hl.scatter(blocks, Q, G)[rank]
    b = blocks[rank]
    for n in range(STEPS):
        if n:
            hl.exchange(blocks, copies, rank, torch.from_numpy(Qb), torch.from_numpy(Gb))
        Qb, Gb, _ = Orc.step(b.grid, b.params, Qb, Gb, dt, eps, 1)
    dist.barrier()
    out.put((rank, Qb, Gb))
    dist.destroy_process_group()


def test_four_gloo_ranks_2x2_periodic():
    """Four ranks in a 2 x 2 block grid, periodic in both directions: every rank exchanges faces
    and corners with the other three (the corner cells of a halo come from the diagonal block)."""
    import torch.multiprocessing as mp
    grid, params, Q, G, dt, eps = problem((I.PERIODIC,) * 4)
    Qu, Gu, _ = O.step(grid, params, Q, G, dt, eps, STEPS)
    blocks = halo.decompose(grid, params, 2, 2, w=2)
    peers = {r: {s for (s, rr) in halo.plan(blocks) if rr == r} for r in range(4)}
    assert all(len(v) == 3 for v in peers.values())
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank2d, args=(r, 4, port, q)) for r in range(4)]
    for p in ps:
        p.start()
    res = sorted((q.get(timeout=240) for _ in range(4)), key=lambda t: t[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    Qs, Gs = np.zeros_like(Q), np.zeros_like(G)
    halo.gather(blocks, [(Qb, Gb) for _, Qb, Gb in res], Qs, Gs)
    assert np.array_equal(Qs, Qu) and np.array_equal(Gs, Gu)


def _rank_exchange_dtypes(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2509_21832_gb300 import halo as hl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    grid = I.Grid(nx=12, ny=6, nv1=4, nv2=3)
    blocks = hl.decompose(grid, I.Params(bc=(I.PERIODIC,) * 4), world, 1, w=2)
    copies = hl.plan(blocks)
    b = blocks[rank]
    gi = torch.as_tensor(b.global_index())
    own = torch.as_tensor(b.owned_mask())
    nc, nv = b.nx * b.ny, grid.nv1 * grid.nv2
    # owned cells carry values made from their global index; halos start as NaN
    Q = (gi[None, :].double() * 10 + torch.arange(6)[:, None]).clone()
    G = (gi[:, None].float() * 100 + torch.arange(nv)[None, :]).clone()
    Q[:, ~own] = float("nan")
    G[~own] = float("nan")
    hl.exchange(blocks, copies, rank, Q.view(6, b.ny, b.nx), G.view(b.ny, b.nx, 3, 4))
    Qx = gi[None, :].double() * 10 + torch.arange(6)[:, None]
    Gx = gi[:, None].float() * 100 + torch.arange(nv)[None, :]
    ok = bool(torch.equal(Q, Qx) and torch.equal(G, Gx) and G.dtype == torch.float32)
    dist.barrier()
    out.put((rank, ok))
    dist.destroy_process_group()


def test_exchange_fills_every_halo_with_the_owners_values_in_their_dtypes():
    """After one exchange every halo cell holds its owner's Q (float64) and g (float32, as FP32 g
    travels), corners and the periodic wrap included."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_exchange_dtypes, args=(r, 3, port, q)) for r in range(3)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(3))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok in res), res
