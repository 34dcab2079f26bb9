"""The closure network trained on the GPU by the library's own kernels, and what it gains over
the plain method: on a held-out bump problem with specular walls the hybrid step must stay within
an L1 density error of 1e-3 of the plain FP64 run while skipping the micro solve in a large part of
the domain, and run faster."""
import numpy as np
import pytest

from paper_2509_21832_gb300 import api
from paper_2509_21832_gb300 import closure
from paper_2509_21832_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(pb, nsteps, mlp=None, thr=None):
    import torch
    with api.Solver(pb.grid, pb.params) as s:
        s.set_state(pb.Q, pb.G)
        if mlp is not None:
            s.set_closure(mlp, thr)
        s.step(pb.dt, pb.eps, 2)  # warm-up of the launch path
        s.set_state(pb.Q, pb.G)
        if mlp is not None:
            s.set_closure(mlp, thr)
        s.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        s.step(pb.dt, pb.eps, nsteps)
        b.record()
        s.sync()
        ms = a.elapsed_time(b)
        Q, _ = s.get_moments()
        frac = None
        if mlp is not None:
            ncl, ncs = s.closure_stats()
            frac = ncl / ncs
    return Q, ms, frac


def test_trained_closure_gain():
    # about 1.3e6 samples from 256^2 x 32^2 runs (five Knudsen numbers, two CFL numbers)
    ds = closure.collect(closure.training_problems(n=256), warm_steps=10, every=12,
                         samples_per_problem=8, keep=0.25)
    assert ds.X.shape[0] >= 10 * 8 * 16384
    res = closure.train(ds, epochs=3, batch=8192, lr=2e-3, lr_final=1e-4, seed=0)
    first, last = res.losses[0][1], res.losses[-1][1]
    print("training: %d samples in %.2f s, %d steps in %.2f s, loss %.4g -> %.4g"
          % (ds.X.shape[0], ds.seconds, res.steps, res.seconds, first, last))
    assert last < 0.2 * first
    # applied on a held-out problem of the 512^2 x 32^2 family
    pb = I.bump_specular(n=512, nv=32, eps=1e-2, seed=7)
    nsteps = 60
    Qp, tp, _ = _run(pb, nsteps)
    Qh, th, frac = _run(pb, nsteps, res.mlp, 1e-3)
    l1 = np.sum(np.abs(Qh[0] - Qp[0])) / np.sum(np.abs(Qp[0]))
    print("512^2 x 32^2, eps 1e-2: plain %.2f ms/step; hybrid %.2f ms/step (x%.2f), closure "
          "fraction %.3f, L1 density error %.3g" % (tp / nsteps, th / nsteps, tp / th, frac, l1))
    assert l1 <= 1e-3
    assert frac >= 0.3
    assert th < tp
    res.mlp.close()
