"""Benchmark of the micro-macro KFVS step on GB300.

Workload: 2D-2V unit box, 256 x 256 cells x 32 x 32 velocities on [-8, 8]^2, specular walls on
all sides, Gaussian density bump (seeded centre), u = 0, T = 1, g = 0, nu = -1/2, tau = rho,
CFL 0.5 (sum form), FP64.  A step is one full time step (prims, micro x sweep, micro y sweep +
relaxation + heat flux, macro x, macro y).  Inputs (two 537 MB FP64 phase-space buffers) are
larger than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--eps E] [--impl reference]

Prints one JSON line (rank 0).  --impl reference times the plain FP64 CPU oracle on this host's
cores on a bounded sample of the same workload (a strip of rows per step).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "phase-space updates/s & %HBM roofline; mixed/learned vs FP64 at set L1 err"
UNIT = "phase-cell updates/s"
# Algorithmic FP64 flops per phase cell of the dominant kernel (y sweep 13, Ghat and blend 15,
# heat-flux moments 8, Maxwellian/Gaussian from separable tables 3) and of the whole step
# (plus the x sweep, 7: the upwind difference, the upwind update and the two projection terms;
# its velocity moments come from row sums of g left by the previous y sweep); algorithmic bytes
# per phase cell and step: one read and one write of g in FP64 plus the per-cell macro fields
# (6 + 6 + 4 + 4 doubles over nv = 1024 velocities).
FLOPS_MICRO_Y = 39.0
FLOPS_STEP = 46.0
BYTES_PER_PHASE_FP64 = 16.0 + 160.0 / 1024.0
# DRAM traffic of k_micro_y per phase cell (32^2 velocity meshes), from an ncu capture of the
# 160^2 x 32^2 bump case: (227.0 MB read, with the row sums and the x sweep's e1, e2, + 190.8 MB
# written) / 26.2144 M phase cells.
TRAFFIC_MICRO_Y_PER_PHASE_CELL = 417.8e6 / 26.2144e6


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# FP64 peak from unit counts and clocks: 152 SMs x 4 FP64 flops/clk/SM (2 FMA) x max SM clock.
def fp64_peak_tflops(sm_max_mhz):
    return 152 * 4 * sm_max_mhz * 1e6 / 1e12


def measure_fp64_peak(stream, reps=5):
    """FP64 pipe throughput measured on this GPU: the library's FMA probe (8 independent chains
    per thread, 8 CTAs of 256 threads per SM, about 0.1 s per launch), best of `reps` launches
    timed with CUDA events on `stream`, in TFLOP/s."""
    import torch
    from paper_2509_21832_gb300 import api
    ctas, iters = 152 * 8, 20000
    out = torch.empty(ctas * 256, dtype=torch.float64, device="cuda")
    best = 0.0
    for r in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = api.mm_diag_fp64_fma(out, ctas, iters, stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        if r > 0:   # the first launch is a warm-up
            best = max(best, flops / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms, pg, device):
    """The slowest rank's time: every rank times the same K steps of its own replica."""
    if pg is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, phase_cells, steps, ms):
    """Whole-job rate of N independent replicas (weak scaling): all ranks' phase-cell updates
    over the slowest rank's time."""
    return world * phase_cells * steps / (ms * 1e-3)


def cpu_baseline(pr, rows, steps):
    """Oracle (as it stands) on this host's cores over a strip of `rows` rows of the workload."""
    from oracle import oracle as O
    from paper_2509_21832_gb300 import inputs as I
    g = pr.grid
    rows = min(rows, g.ny)
    dy = (g.y1 - g.y0) / g.ny
    sub = I.Grid(nx=g.nx, ny=rows, x0=g.x0, x1=g.x1, y0=g.y0, y1=g.y0 + rows * dy, nv1=g.nv1,
                 nv2=g.nv2, v1min=g.v1min, v1max=g.v1max, v2min=g.v2min, v2max=g.v2max)
    Q = np.ascontiguousarray(pr.Q[:, :rows])
    G = np.ascontiguousarray(pr.G[:rows])
    t0 = time.perf_counter()
    O.step(sub, pr.params, Q, G, pr.dt, pr.eps, steps)
    t = time.perf_counter() - t0
    return sub.nphase * steps / t, t, O.num_threads(), sub


def run_reference(args, pr, world, rank):
    if rank != 0:
        return
    from oracle import build as obuild
    obuild.build()
    rows = args.ref_rows
    # warm-up steps (untimed), then K timed steps, each one oracle step over the strip
    if args.warmup > 0:
        cpu_baseline(pr, rows, args.warmup)
    value, t, cores, sub = cpu_baseline(pr, rows, args.steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(pr, args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d steps of a %dx%d-row strip (%d phase cells) of the "
                                   "workload" % (args.steps, sub.nx, sub.ny, sub.nphase)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(pr, args):
    g = pr.grid
    return {"workload": "bump_specular_%dx%dx%dx%d_fp64" % (g.nx, g.ny, g.nv1, g.nv2),
            "nx": g.nx, "ny": g.ny, "nv1": g.nv1, "nv2": g.nv2, "eps": pr.eps,
            "dt": pr.dt, "bc": "specular x4", "nu": pr.params.nu, "tau": "rho",
            "seed": pr.meta.get("seed"),
            "l2": "inputs larger than L2: two %d MB FP64 phase-space buffers" % (g.nphase * 8 // 2**20),
            "parallelism": "replicas" if args.gpus > 1 else "single"}


def plain_variant(pr, stream, steps, oracle_rows, oracle_steps, name, compare=False):
    """A plain FP64 workload other than the headline one: device-resident throughput over
    `steps` steps (CUDA events on the context stream, per-kernel timing off), and the oracle as
    it stands on this host's cores over `oracle_steps` steps of a strip of `oracle_rows` rows.
    With compare, the oracle runs the same full problem and the line carries the largest
    relative difference of the macro fields (max over cells of |Q_gpu - Q_oracle| over
    max(max |Q_oracle,c|, max rho), per component)."""
    import torch
    from paper_2509_21832_gb300 import api
    s = api.Solver(pr.grid, pr.params, stream=stream.cuda_stream)
    s.set_state(pr.Q, pr.G)
    s.step(pr.dt, pr.eps, 3)
    s.sync()
    s.set_state(pr.Q, pr.G)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(pr.dt, pr.eps, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    Qg, _ = s.get_moments(with_H=False)
    s.close()
    nph = pr.grid.nphase
    cv, ct, cores, sub = cpu_baseline(pr, oracle_rows, oracle_steps)
    out = {"variant": name, "eps": pr.eps, "steps": steps, "dtype": "f64",
           "value": nph * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
           "phase_cells": nph,
           "cpu_baseline": {"value": cv, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "%d steps of a %dx%d-row strip (%d phase cells), %.1f s"
                                      % (oracle_steps, sub.nx, sub.ny, sub.nphase, ct)}}
    if compare and sub.ny == pr.grid.ny and oracle_steps == steps:
        from oracle import oracle as O
        Qo, _, _ = O.step(pr.grid, pr.params, pr.Q, pr.G, pr.dt, pr.eps, steps)
        scale = np.maximum(np.max(np.abs(Qo), axis=(1, 2)), np.max(Qo[0]))
        out["max_rel_err_vs_oracle"] = float(np.max(np.max(np.abs(Qg - Qo), axis=(1, 2)) / scale))
    return out


def fp32_variant(args, stream):
    """Four-quadrant Riemann data, diffuse bottom wall, 1024^2 x 24^2, g in FP32: throughput,
    HBM fraction (8 algorithmic bytes per phase cell: one FP32 read and write of g) and the
    relative L1 density error against the FP64 path after the same number of steps."""
    import torch
    from paper_2509_21832_gb300 import api
    from paper_2509_21832_gb300 import inputs as I
    pr = I.riemann4_diffuse(n=args.variant_n, nv=24, eps=1e-2, seed=0, nsteps=100)
    out = {"workload": "riemann4_diffuse_%dx%dx24x24" % (pr.grid.nx, pr.grid.ny),
           "eps": pr.eps, "steps": pr.nsteps, "dtype": "g f32 (transport, velocity sums, relaxation); ES tensor inverse, heat-flux totals, macro update f64"}
    res = {}
    for prec in (I.PREC_G_FP32, I.PREC_FP64):
        params = I.Params(**{**pr.params.__dict__, "precision": prec})
        s = api.Solver(pr.grid, params, stream=stream.cuda_stream)
        s.set_state(pr.Q, None)
        s.step(pr.dt, pr.eps, 3)
        s.sync()
        s.set_state(pr.Q, None)
        s.set_timing(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(pr.dt, pr.eps, pr.nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kt = s.get_timing()
        Q, _ = s.get_moments(with_H=False)
        s.close()
        res[prec] = (ms, kt, Q)
    ms, kt, Q32 = res[I.PREC_G_FP32]
    ms64, _, Q64 = res[I.PREC_FP64]
    nph = pr.grid.nphase
    peaks, src = measured_peaks()
    hbm = (8.0 + 160.0 / 576.0) * nph * pr.nsteps / (ms * 1e-3) / 1e9
    out.update({
        "value": nph * pr.nsteps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / pr.nsteps,
        "fp64_ms_per_step": ms64 / pr.nsteps, "speedup_vs_fp64": ms64 / ms,
        "hbm_achieved_gbs": hbm, "hbm_frac": hbm / peaks["hbm_gbs"],
        "l1_density_rel_err_vs_fp64": float(np.sum(np.abs(Q32[0] - Q64[0])) / np.sum(np.abs(Q64[0]))),
        # per step, summed over the launches of a kind (the phase-space kernel is launched once
        # per group of row segments)
        "kernel_ms_per_step": {k: v[0] / pr.nsteps for k, v in kt.items() if v[1]},
        "launches_per_step": {k: v[1] / pr.nsteps for k, v in kt.items() if v[1]}})
    return out


def closure_variant(args, stream):
    """Learned closure on the bump family with specular walls: the network is trained on the
    GPU (library kernels) from about 1.3e6 samples of 256^2 x 32^2 plain runs, then the hybrid
    step is timed against the plain FP64 step on 512^2 x 32^2 at eps = 1e-3, 1e-2 and 1e-1
    (indicator thresholds 1e-3 and 1e-2), with the relative L1 density error of the hybrid run
    against the plain run after the same steps.  value = phase cells x steps / time of the hybrid run (an equivalent
    rate: closure cells do not advance g)."""
    import torch
    from paper_2509_21832_gb300 import api, closure
    from paper_2509_21832_gb300 import inputs as I
    ds = closure.collect(closure.training_problems(n=256), warm_steps=10, every=12,
                         samples_per_problem=8, keep=0.25)
    res = closure.train(ds, epochs=3, batch=8192, lr=2e-3, lr_final=1e-4, seed=0)
    out = {"workload": "bump_specular_%dx%dx32x32_learned_closure" % (args.closure_n, args.closure_n),
           "threshold": 1e-3, "steps": args.closure_steps, "dtype": "f64 (network bf16/f32)",
           "training": {"samples": int(ds.X.shape[0]), "collect_s": ds.seconds,
                        "adam_steps": res.steps, "train_s": res.seconds,
                        "train_samples_per_s": 3 * int(ds.X.shape[0]) / res.seconds,
                        "kernels": "forward/backward and weight gradients on the tensor cores "
                                   "(mma m16n8k16, BF16 operands, FP32 accumulation)",
                        "loss_first": res.losses[0][1], "loss_last": res.losses[-1][1]},
           "cases": []}

    def run(pb, mlp, thr):
        s = api.Solver(pb.grid, pb.params, stream=stream.cuda_stream)
        s.set_state(pb.Q, pb.G)
        if mlp is not None:
            s.set_closure(mlp, thr)
        s.step(pb.dt, pb.eps, 3)
        s.set_state(pb.Q, pb.G)
        if mlp is not None:
            s.set_closure(mlp, thr)
        s.set_timing(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(pb.dt, pb.eps, args.closure_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kt = s.get_timing()
        Q, _ = s.get_moments(with_H=False)
        frac, modes = None, None
        if mlp is not None:
            ncl, ncs = s.closure_stats()
            frac = ncl / ncs
            modes = s.closure_steps()
        s.close()
        return ms, kt, Q, frac, modes

    for eps in (1e-3, 1e-2, 1e-1):
        pb = I.bump_specular(n=args.closure_n, nv=32, eps=eps, seed=7)
        msp, ktp, Qp, _, _ = run(pb, None, 1e-3)
        for thr in (1e-3, 1e-2):
            msh, kt, Qh, frac, modes = run(pb, res.mlp, thr)
            nst = args.closure_steps
            out["cases"].append({
                "eps": eps, "threshold": thr, "plain_ms_per_step": msp / nst,
                "hybrid_ms_per_step": msh / nst, "speedup_vs_fp64": msp / msh,
                "closure_fraction": frac, "hybrid_steps": modes[0], "plain_fallback_steps": modes[1],
                "value": pb.grid.nphase * nst / (msh * 1e-3),
                "unit": UNIT,
                "l1_density_rel_err_vs_fp64": float(np.sum(np.abs(Qh[0] - Qp[0])) / np.sum(np.abs(Qp[0]))),
                "kernel_ms": {k: v[0] / v[1] for k, v in kt.items() if v[1]},
                "plain_kernel_ms": {k: v[0] / v[1] for k, v in ktp.items() if v[1]}})
    res.mlp.close()
    return out


def batch_variant(args, count=None, nmin=64, nmax=256, steps=None):
    """count independent periodic problems (cells per side U{nmin..nmax}, velocity meshes
    16^2..32^2, eps log-uniform on [1e-3, 1], seeded Fourier-mode fields; by default the 64
    problems of 64..256 cells per side), stepped as one batch: every call of K steps is one
    persistent launch walking a work queue of (step, problem, phase, tile) items, replayed as a
    CUDA graph, with autotuned tiles.  FP64.  Compared with stepping the same problems through
    separate single-problem contexts, one after the other."""
    import torch
    from paper_2509_21832_gb300 import api
    from paper_2509_21832_gb300 import inputs as I
    count = args.batch_count if count is None else count
    probs = I.batch_problems(count=count, seed=0, nmin=nmin, nmax=nmax)
    nph = sum(p.grid.nphase for p in probs)
    dts = [p.dt for p in probs]
    epss = [p.eps for p in probs]
    steps = args.batch_steps if steps is None else steps
    b = api.BatchSolver([p.grid for p in probs], [p.params for p in probs])
    for q, p in enumerate(probs):
        b.set_state(q, p.Q, None)
    b.step(dts, epss, 1)
    for q, p in enumerate(probs):
        b.set_state(q, p.Q, None)
    threads, ctas = b.autotune()
    tiles = b.tiles()
    b.step(dts, epss, 2)
    b.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(dts, epss, steps)
    b.sync()
    tb = time.perf_counter() - t0
    b.close()
    # the same problems, one context each, stepped one after the other
    ss = [api.Solver(p.grid, p.params) for p in probs]
    for s_, p in zip(ss, probs):
        s_.set_state(p.Q, None)
        s_.step(p.dt, p.eps, 1)
    for s_ in ss:
        s_.sync()
    n_sep = max(1, steps // 10)
    t0 = time.perf_counter()
    for _ in range(n_sep):
        for s_, p in zip(ss, probs):
            s_.step(p.dt, p.eps, 1)
    for s_ in ss:
        s_.sync()
    tsep = (time.perf_counter() - t0) / n_sep
    for s_ in ss:
        s_.close()
    return {"workload": "batch_%d_periodic_problems_%d_to_%d_cells_per_side"
                        % (len(probs), nmin, nmax), "phase_cells": nph,
            "steps": steps, "dtype": "f64", "value": nph * steps / tb, "unit": UNIT,
            "ms_per_step": 1e3 * tb / steps,
            "autotuned": {"threads": threads, "ctas": ctas, "cells_per_micro_item": tiles[0],
                          "cells_per_cell_item": tiles[1]},
            "launches_per_call": 1,
            "separate_contexts_ms_per_step": 1e3 * tsep,
            "speedup_vs_separate_contexts": tsep / (tb / steps)}


def run_blocks(pr, world, rank, steps, warmup, make_stepper, device, group=None):
    """One problem split into px x py spatial blocks, one per rank (Section 5.5's decomposition):
    each rank steps its block (owned cells and a halo of two cells on every side that borders
    another block), refreshing the halos from their owners before every step with point-to-point
    messages over torch.distributed (NCCL between GPUs, gloo on CPU; no collective).
    make_stepper(pr, block, Q, G) returns step(regions) that advances the block's tensors one step
    in place, told which regions of g the exchange rewrote.  Returns (block, Q, G, seconds of
    the timed steps on this rank)."""
    import torch
    import torch.distributed as dist
    from paper_2509_21832_gb300 import halo
    px, py = halo.block_shape(world)
    blocks = halo.decompose(pr.grid, pr.params, px, py, w=2)
    copies = halo.plan(blocks)
    b = blocks[rank]
    Qb, Gb = halo.scatter(blocks, pr.Q, pr.G)[rank]
    Qt = torch.from_numpy(np.ascontiguousarray(Qb)).to(device)
    Gt = torch.from_numpy(np.ascontiguousarray(Gb)).to(device)
    step = make_stepper(pr, b, Qt, Gt)
    regions = halo.halo_regions(b)
    cuda = Qt.is_cuda

    def one():
        halo.exchange(blocks, copies, rank, Qt, Gt, group=group)
        step(regions)

    sync = dist.is_available() and dist.is_initialized()
    for _ in range(warmup):
        one()
    if cuda:
        torch.cuda.synchronize()
    if sync:
        dist.barrier(group=group)
    t0 = time.perf_counter()
    if cuda:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
    for _ in range(steps):
        one()
    if cuda:
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
    else:
        sec = time.perf_counter() - t0
    if sync:
        dist.barrier(group=group)
    return b, Qt, Gt, sec


def gpu_block_stepper(pr, b, Qt, Gt):
    """The library on the block's own CUDA tensors (a borrowed context on torch's current
    stream, which also carries the halo copies)."""
    import torch
    from paper_2509_21832_gb300 import api
    S = torch.empty(api.mm_scratch_bytes(b.grid, b.params), dtype=torch.uint8, device=Qt.device)
    s = api.Solver(b.grid, b.params, stream=torch.cuda.current_stream().cuda_stream,
                   borrow=(Qt, Gt, S))
    s.scratch = S
    s.set_state(Qt.clone(), Gt.clone())

    def step(regions):
        for r in regions:
            s.g_region_changed(*r)
        s.step(pr.dt, pr.eps, 1)

    step.solver = s
    return step


def summarize_variant(v):
    """The headline line's short form of a variant (its full line is printed before it)."""
    keep = ("value", "ms_per_step", "speedup_vs_fp64", "hbm_frac", "l1_density_rel_err_vs_fp64",
            "speedup_vs_separate_contexts", "max_rel_err_vs_oracle", "steps", "eps")
    out = {k: v[k] for k in keep if k in v}
    if "cpu_baseline" in v:
        out["cpu_baseline_value"] = v["cpu_baseline"]["value"]
    if "training" in v:
        out["train_samples_per_s"] = v["training"]["train_samples_per_s"]
    if "cases" in v:
        out["cases"] = [{k: c[k] for k in ("eps", "threshold", "speedup_vs_fp64",
                                           "closure_fraction", "plain_fallback_steps",
                                           "l1_density_rel_err_vs_fp64")}
                        for c in v["cases"]]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--eps", type=float, default=1e-1)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--nv", type=int, default=32)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--ref-rows", type=int, default=32)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--variant-n", type=int, default=1024)
    ap.add_argument("--variant-only", action="store_true")
    ap.add_argument("--batch-only", action="store_true")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=100)
    ap.add_argument("--batch-nmin", type=int, default=64)
    ap.add_argument("--batch-nmax", type=int, default=256)
    ap.add_argument("--closure-only", action="store_true")
    ap.add_argument("--closure-n", type=int, default=512)
    ap.add_argument("--closure-steps", type=int, default=100)
    ap.add_argument("--decompose", action="store_true",
                    help="split the one problem into spatial blocks, one per rank (halo exchange "
                         "between ranks every step) instead of running one replica per rank")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from paper_2509_21832_gb300 import inputs as I
    pr = I.bump_specular(n=args.n, nv=args.nv, eps=args.eps, seed=0)
    world, rank, local = dist_setup(args)

    if args.impl == "reference":
        run_reference(args, pr, world, rank)
        return
    if args.batch_only:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps(batch_variant(args, nmin=args.batch_nmin, nmax=args.batch_nmax)),
              flush=True)
        print(json.dumps(batch_variant(args, count=256, nmin=16, nmax=48, steps=50)), flush=True)
        return
    if args.variant_only:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps(fp32_variant(args, torch.cuda.Stream())), flush=True)
        return
    if args.closure_only:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps(closure_variant(args, torch.cuda.Stream())), flush=True)
        return

    import torch
    from paper_2509_21832_gb300 import api

    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    if args.decompose:
        b, _, _, sec = run_blocks(pr, world, rank, args.steps, args.warmup, gpu_block_stepper,
                                  torch.device("cuda", local))
        ms = max_over_ranks(1e3 * sec, pg, "cuda")
        if rank == 0:
            from paper_2509_21832_gb300 import halo
            px, py = halo.block_shape(world)
            cfg = dict(config_of(pr, args), parallelism="spatial blocks %dx%d, halo 2" % (px, py))
            print(json.dumps({
                "metric": METRIC, "value": pr.grid.nphase * args.steps / (ms * 1e-3),
                "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg}),
                flush=True)
        if pg:
            pg.destroy_process_group()
        return

    stream = torch.cuda.Stream()
    solver = api.Solver(pr.grid, pr.params, stream=stream.cuda_stream)
    Qd = torch.from_numpy(pr.Q).cuda()
    Gd = torch.zeros(pr.grid.nphase, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    solver.set_state(Qd, Gd)
    for _ in range(args.warmup):
        solver.step(pr.dt, pr.eps, 1)
    solver.sync()

    def timed_run(K, timing):
        solver.set_timing(timing)
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.3)
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            solver.step(pr.dt, pr.eps, 1)
        e1.record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        sampler.stop()
        solver.sync()
        ms = e0.elapsed_time(e1)
        kt = solver.get_timing() if timing else None
        solver.set_timing(False)
        return ms, kt, sampler.summary()

    # the headline: K steps with the library's per-kernel events off
    ms, _, clocks = timed_run(args.steps, False)
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if set(clocks["reasons"]) & bad:
        ms, _, clocks = timed_run(args.steps, False)
    ms = max_over_ranks(ms, pg, "cuda")
    nph = pr.grid.nphase
    value = replica_value(world, nph, args.steps, ms)
    # the per-kernel split (and the roofline's kernel duration): the same K steps again with an
    # event pair around every launch, on the context stream that the kernels run on
    ms_split, kt, clocks_split = timed_run(args.steps, True)
    launches = sum(n for (_, n) in kt.values())

    peaks, peak_src = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp64_units = fp64_peak_tflops(sm_max)
    fp64_peak = measure_fp64_peak(stream)
    ky_ms, ky_n = kt["micro_y"]
    achieved = FLOPS_MICRO_Y * nph / (ky_ms / ky_n * 1e-3) / 1e12
    hbm_gbs = BYTES_PER_PHASE_FP64 * nph * args.steps / (ms * 1e-3) / 1e9
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak,
                # DRAM bytes per k_micro_y launch: ncu capture of the 160^2 x 32^2 case
                # (read + write = 417.8 MB over 26.2 M phase cells), scaled by phase cells
                "traffic": (TRAFFIC_MICRO_Y_PER_PHASE_CELL * nph
                            if (pr.grid.nv1, pr.grid.nv2) == (32, 32) else None),
                "traffic_unit": "bytes per launch",
                "kernel": "micro_y",
                "peak_source": "measured: FP64 FMA probe (mm_diag_fp64_fma), best of 5 launches "
                               "on this GPU; unit counts give %.3f TFLOP/s (152 SMs x 4 flop/clk "
                               "x %.0f MHz)" % (fp64_units, sm_max),
                "split_run_ms_per_step": ms_split / args.steps,
                "step_fp64_frac": FLOPS_STEP * nph * args.steps / (ms * 1e-3) / 1e12 / fp64_peak,
                "hbm_achieved_gbs": hbm_gbs, "hbm_peak_gbs": peaks["hbm_gbs"],
                "hbm_frac": hbm_gbs / peaks["hbm_gbs"], "hbm_peak_source": peak_src,
                "kernel_ms": {k: (v[0] / v[1] if v[1] else None) for k, v in kt.items()}}

    # end to end through the C ABI with pinned host buffers: every step takes (Q, G) from host
    # memory and returns (Q, H) to it (mm_step_host: the copy of G overlapped with the step)
    e2e = None
    if args.e2e_steps > 0:
        Qh = torch.from_numpy(pr.Q.copy()).pin_memory().numpy()
        Gh = torch.zeros(nph, dtype=torch.float64).pin_memory().numpy()
        Qo = torch.empty(6 * pr.grid.ncell, dtype=torch.float64).pin_memory().numpy()
        Ho = torch.empty(4 * pr.grid.ncell, dtype=torch.float64).pin_memory().numpy()
        Qo = Qo.reshape(6, pr.grid.ny, pr.grid.nx)
        Ho = Ho.reshape(4, pr.grid.ny, pr.grid.nx)
        for _ in range(2):
            solver.step_host(Qh, Gh, pr.dt, pr.eps, Qo, Ho)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            solver.step_host(Qh, Gh, pr.dt, pr.eps, Qo, Ho)
        t = time.perf_counter() - t0
        e2e = {"value": world * nph * args.e2e_steps / t, "unit": UNIT,
               "h2d_bytes_per_step": int(Qh.nbytes + Gh.nbytes),
               "d2h_bytes_per_step": int(Qo.nbytes + Ho.nbytes),
               "steps": args.e2e_steps,
               "api": "mm_step_host (host (Q, G) in, host (Q, H) out, every step)"}
    solver.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # calibrate on one step of the full grid, then time enough steps for ~12 s of wall time
        _, t1, _, _ = cpu_baseline(pr, pr.grid.ny, 1)
        n = max(1, min(100, int(round(12.0 / max(t1, 1e-3)))))
        v, t, cores, sub = cpu_baseline(pr, pr.grid.ny, n)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d steps of the full %dx%d grid (%d phase cells), %.1f s"
                         % (n, sub.nx, sub.ny, sub.nphase, t)}

    variants = None
    if rank == 0 and not args.no_variants:
        full = {
            # the 1D-2V Sod shock tube (200 x 24^2, 640 steps to t = 0.2), checked against the
            # oracle's full run on this host
            "sod_1d2v_200x24x24_fp64": plain_variant(I.sod_1d2v(), stream, 640, 1, 640,
                                                      "sod_1d2v_200x24x24_fp64", compare=True),
            # the headline workload at the other Knudsen number of its family
            "bump_specular_256x256x32x32_eps1e-3_fp64": plain_variant(
                I.bump_specular(n=args.n, nv=args.nv, eps=1e-3, seed=0), stream, args.steps, 32,
                8, "bump_specular_256x256x32x32_eps1e-3_fp64"),
            "riemann4_diffuse_1024x1024x24x24_fp32g": fp32_variant(args, stream),
            "batch_64_periodic_fp64": batch_variant(args),
            # where batching matters: many problems too small to fill the GPU alone
            "batch_256_small_periodic_fp64": batch_variant(args, count=256, nmin=16, nmax=48,
                                                           steps=50),
            "bump_specular_512x512x32x32_learned_closure": closure_variant(args, stream)}
        for k, v in full.items():
            print(json.dumps(dict(v, variant=k)), flush=True)
        variants = {k: summarize_variant(v) for k, v in full.items()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "config": config_of(pr, args),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks, "variants": variants}
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
