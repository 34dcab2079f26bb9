"""Learned heat-flux closure: training data from plain runs, normalisation, and training of the
closure network on the GPU with the library's own kernels (mm_mlp_*).

The closure is an extension of the library (the paper has no learned closure).  The network maps
39 local features of a cell (mm_closure_features) to y = (H - H_CE) / (eps rho T^{3/2}), the part
of the heat flux of Eq. (5-99) beyond its Chapman-Enskog value.  Training data are (features of
Q^n, target after one plain micro-macro step) pairs collected on the device by
mm_closure_collect; the loss is the mean squared error of the standardised outputs and the
optimiser Adam on FP32 master weights with BF16 copies for the kernels.  This module only
arranges buffers and calls; every forward, backward and update runs in the library's kernels.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import api
from . import inputs as I


@dataclass
class Dataset:
    X: "torch.Tensor"   # [n][39] float32, CUDA
    Y: "torch.Tensor"   # [n][4] float32, CUDA
    seconds: float = 0.0


def collect(problems, warm_steps: int, every: int, samples_per_problem: int, keep: float = 1.0,
            seed: int = 0, device="cuda"):
    """Run each problem with the plain solver; after warm_steps, every `every` steps record the
    features of Q^n and the target of the next step, samples_per_problem times, keeping a seeded
    random fraction `keep` of the cells of each snapshot.

    problems: iterable of inputs.Problem (FP64).  Returns a Dataset on the device."""
    import torch
    Xs, Ys = [], []
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    t0 = time.time()
    for pb in problems:
        nc = pb.grid.nx * pb.grid.ny
        with api.Solver(pb.grid, pb.params) as s:
            s.set_state(pb.Q, pb.G)
            if warm_steps > 0:
                s.step(pb.dt, pb.eps, warm_steps)
            for _ in range(samples_per_problem):
                X = torch.empty((nc, api.MLP_IN), dtype=torch.float32, device=device)
                Y = torch.empty((nc, api.MLP_OUT), dtype=torch.float32, device=device)
                s.closure_collect(pb.dt, pb.eps, X, Y)
                if keep < 1.0:
                    idx = torch.randperm(nc, device=device, generator=gen)[:max(1, int(keep * nc))]
                    X, Y = X.index_select(0, idx), Y.index_select(0, idx)
                Xs.append(X)
                Ys.append(Y)
                if every > 1:
                    s.step(pb.dt, pb.eps, every - 1)
            s.sync()
    torch.cuda.synchronize()
    return Dataset(torch.cat(Xs), torch.cat(Ys), time.time() - t0)


def normalisation(ds: Dataset) -> np.ndarray:
    """[x mean, x 1/std, y mean, y std] of a dataset (features with zero spread get 1/std = 1)."""
    X = ds.X.double()
    Y = ds.Y.double()
    mx, sx = X.mean(0), X.std(0)
    my, sy = Y.mean(0), Y.std(0)
    isx = 1.0 / sx.clamp_min(1e-12)
    isx[sx <= 1e-12] = 1.0
    sy = sy.clamp_min(1e-12)
    return np.concatenate([mx.cpu().numpy(), isx.cpu().numpy(), my.cpu().numpy(),
                           sy.cpu().numpy()]).astype(np.float32)


def initial_params(seed: int) -> np.ndarray:
    """Kaiming-normal weights for the GELU layers (std sqrt(2/fan_in)), 1/fan_in variance for the
    linear output layer, zero biases."""
    rng = np.random.default_rng(seed)
    h, i, o = api.MLP_HIDDEN, api.MLP_IN, api.MLP_OUT
    parts = [rng.normal(0.0, math.sqrt(2.0 / i), h * i), np.zeros(h),
             rng.normal(0.0, math.sqrt(2.0 / h), h * h), np.zeros(h),
             rng.normal(0.0, math.sqrt(1.0 / h), o * h), np.zeros(o)]
    return np.concatenate(parts).astype(np.float32)


@dataclass
class TrainResult:
    mlp: "api.MLP"
    norm: np.ndarray
    losses: list
    steps: int
    seconds: float


def train(ds: Dataset, epochs: int = 4, batch: int = 8192, lr: float = 2e-3, seed: int = 0,
          lr_final: float = 2e-4, log_every: int = 50) -> TrainResult:
    """Adam on mini-batches of a shuffled dataset, learning rate decayed geometrically from lr to
    lr_final; returns the trained network and the loss every log_every steps."""
    import torch
    norm = normalisation(ds)
    mlp = api.MLP(initial_params(seed), norm)
    n = ds.X.shape[0]
    nb = max(1, n // batch)
    total = epochs * nb
    gen = torch.Generator(device=ds.X.device)
    gen.manual_seed(seed)
    losses = []
    t0 = time.time()
    step = 0
    for _ in range(epochs):
        perm = torch.randperm(n, device=ds.X.device, generator=gen)
        Xp = ds.X.index_select(0, perm)
        Yp = ds.Y.index_select(0, perm)
        for b in range(nb):
            lr_t = lr * (lr_final / lr) ** (step / max(1, total - 1))
            want = step % log_every == 0 or step == total - 1
            L = mlp.train_step(Xp[b * batch:(b + 1) * batch], Yp[b * batch:(b + 1) * batch], lr_t,
                               want_loss=want)
            if want:
                losses.append((step, L))
            step += 1
    torch.cuda.synchronize()
    return TrainResult(mlp, norm, losses, step, time.time() - t0)


def training_problems(n: int = 256, nv: int = 32, eps_list=(1e-3, 3e-3, 1e-2, 3e-2, 1e-1),
                      cfls=(0.5, 0.25), seed: int = 11):
    """Bump problems with specular walls (the family the closure is applied to) over a range of
    Knudsen numbers and two CFL numbers (so that the relaxation weight omega1 = eps/(eps + dt tau)
    of finer meshes is covered), as training runs."""
    out = []
    for k, eps in enumerate(eps_list):
        for m, cfl in enumerate(cfls):
            out.append(I.bump_specular(n=n, nv=nv, eps=eps, seed=seed + 100 * k + m, cfl=cfl))
    return out
