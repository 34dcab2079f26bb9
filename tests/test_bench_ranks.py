"""The benchmark's multi-rank logic on CPU: two gloo ranks combine their times as the maximum
and report the whole-job rate of independent replicas; the reference arm prints from rank 0
only."""
import json
import os
import socket
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(times[rank], dist, "cpu")
    val = bench.replica_value(world, 1000, 10, ms)
    dist.barrier()
    out.put((rank, ms, val))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [12.5, 20.0]
    ps = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, val in res:
        assert ms == 20.0
        assert val == 2 * 1000 * 10 / 20e-3


def _torchrun(args, nproc=2, timeout=300):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           "--nproc-per-node", str(nproc), "--master-addr", "127.0.0.1",
           "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py")] + args
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_line_from_rank_0():
    r = _torchrun(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
                   "--nv", "8", "--ref-rows", "2"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def _oracle_stepper(pr, b, Qt, Gt):
    """Steps a block's CPU tensors in place with the oracle (the test's stand-in for the library
    on a GPU)."""
    from oracle import oracle as O

    def step(regions):
        Q, G, _ = O.step(b.grid, b.params, Qt.numpy(), Gt.numpy(), pr.dt, pr.eps, 1)
        Qt.numpy()[...] = Q
        Gt.numpy()[...] = G

    return step


def _decomposed_worker(rank, world, port, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist
    import bench
    from paper_2509_21832_gb300 import inputs as I
    from test_bench_ranks import _oracle_stepper
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pr = I.bump_specular(n=12, nv=8, eps=1e-2, seed=3)
    b, Qt, Gt, sec = bench.run_blocks(pr, world, rank, steps, 0, _oracle_stepper,
                                      torch.device("cpu"))
    ms = bench.max_over_ranks(1e3 * sec, dist, "cpu")
    out.put((rank, Qt.numpy().copy(), Gt.numpy().copy(), ms))
    dist.destroy_process_group()


def test_decomposed_bench_entry_reproduces_the_undivided_run_on_gloo_ranks():
    """bench.run_blocks, the entry of `bench.py --decompose`, on two gloo ranks (the oracle
    stepping each rank's block, faces exchanged point to point every step): the owned cells of
    both blocks equal the undivided oracle run bit for bit, and both ranks report the same (max)
    time."""
    import numpy as np
    import torch.multiprocessing as mp
    from oracle import oracle as O
    from paper_2509_21832_gb300 import halo
    from paper_2509_21832_gb300 import inputs as I
    steps = 3
    pr = I.bump_specular(n=12, nv=8, eps=1e-2, seed=3)
    Qu, Gu, _ = O.step(pr.grid, pr.params, pr.Q, pr.G, pr.dt, pr.eps, steps)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_decomposed_worker, args=(r, 2, port, steps, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(2)), key=lambda t: t[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    blocks = halo.decompose(pr.grid, pr.params, 2, 1, w=2)
    Qs, Gs = np.zeros_like(Qu), np.zeros_like(Gu)
    halo.gather(blocks, [(Qb, Gb) for _, Qb, Gb, _ in res], Qs, Gs)
    assert np.array_equal(Qs, Qu) and np.array_equal(Gs, Gu)
    assert res[0][3] == res[1][3] > 0
    assert halo.block_shape(2) == (2, 1) and halo.block_shape(8) == (4, 2)
