"""Plain FP64 reference of the learned heat-flux closure network (test infrastructure only).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the CPU-baseline leg
of the benchmark; the product path never uses it.  It shares no code with the CUDA library.

The network is the library's extension (the paper has no learned closure): a multilayer
perceptron with 39 inputs, two hidden layers of 64 GELU units and 4 outputs.  Parameters are one
flat vector [W1 (64x39, row-major by output unit), b1 (64), W2 (64x64), b2 (64), W3 (4x64),
b3 (4)] of 6980 values; the normalisation vector is [input mean (39), input 1/std (39), output
mean (4), output std (4)].  With x' = (x - mean_x) / std_x,

    a1 = gelu(W1 x' + b1),  a2 = gelu(W2 a1 + b2),  y' = W3 a2 + b3,  y = y' std_y + mean_y,

and training minimises L = (1/n) sum_s sum_o (y'_so - t'_so)^2 with t' = (t - mean_y) / std_y.
gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2 (the exact form).  The kernels store the
weights in BF16 and accumulate in FP32; this reference evaluates the same BF16-rounded weights in
FP64 so that the two differ only by the kernels' FP32 arithmetic.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

N_IN, N_HIDDEN, N_OUT = 39, 64, 4
OFF_W1 = 0
OFF_B1 = OFF_W1 + N_HIDDEN * N_IN
OFF_W2 = OFF_B1 + N_HIDDEN
OFF_B2 = OFF_W2 + N_HIDDEN * N_HIDDEN
OFF_W3 = OFF_B2 + N_HIDDEN
OFF_B3 = OFF_W3 + N_OUT * N_HIDDEN
N_PARAM = OFF_B3 + N_OUT


def bf16_round(w) -> np.ndarray:
    """Round FP32 values to the nearest BF16 value (ties to even), returned as FP64.

    BF16 keeps the sign, the 8 exponent bits and the top 7 mantissa bits of an FP32 number; the
    rounding adds half an ulp of the kept part (minus one when the kept part is even) to the
    discarded 16 bits and truncates."""
    f = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = ((bits + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return bits.view(np.float32).astype(np.float64)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    W1 = p[OFF_W1:OFF_B1].reshape(N_HIDDEN, N_IN)
    b1 = p[OFF_B1:OFF_W2]
    W2 = p[OFF_W2:OFF_B2].reshape(N_HIDDEN, N_HIDDEN)
    b2 = p[OFF_B2:OFF_W3]
    W3 = p[OFF_W3:OFF_B3].reshape(N_OUT, N_HIDDEN)
    b3 = p[OFF_B3:N_PARAM]
    return W1, b1, W2, b2, W3, b3


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _forward(params, norm, X):
    W1, b1, W2, b2, W3, b3 = unpack(params)
    norm = np.asarray(norm, dtype=np.float64)
    mx, isx = norm[:N_IN], norm[N_IN:2 * N_IN]
    xs = (np.asarray(X, dtype=np.float64) - mx) * isx
    z1 = xs @ W1.T + b1
    a1 = gelu(z1)
    z2 = a1 @ W2.T + b2
    a2 = gelu(z2)
    ys = a2 @ W3.T + b3
    return xs, z1, a1, z2, a2, ys


def forward(params, norm, X) -> np.ndarray:
    """Network output y (de-standardised) for samples X [n][39]."""
    norm = np.asarray(norm, dtype=np.float64)
    ys = _forward(params, norm, X)[-1]
    return ys * norm[2 * N_IN + N_OUT:] + norm[2 * N_IN:2 * N_IN + N_OUT]


def loss(params, norm, X, T) -> float:
    norm = np.asarray(norm, dtype=np.float64)
    ys = _forward(params, norm, X)[-1]
    ts = (np.asarray(T, dtype=np.float64) - norm[2 * N_IN:2 * N_IN + N_OUT]) / norm[2 * N_IN + N_OUT:]
    return float(np.sum((ys - ts) ** 2) / len(ys))


def loss_and_grad(params, norm, X, T):
    """Loss and its gradient with respect to the parameters, by the chain rule layer by layer."""
    norm = np.asarray(norm, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(params)
    xs, z1, a1, z2, a2, ys = _forward(params, norm, X)
    n = len(ys)
    ts = (np.asarray(T, dtype=np.float64) - norm[2 * N_IN:2 * N_IN + N_OUT]) / norm[2 * N_IN + N_OUT:]
    e = ys - ts
    L = float(np.sum(e * e) / n)
    d3 = 2.0 * e / n                      # dL/dy'
    gW3 = d3.T @ a2
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ W3) * gelu_grad(z2)        # dL/dz2
    gW2 = d2.T @ a1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * gelu_grad(z1)        # dL/dz1
    gW1 = d1.T @ xs
    gb1 = d1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def loss_and_grad_bf16(params, norm, X, T, rnd=None):
    """Loss and gradient as the training kernels form them: the same chain rule as
    loss_and_grad, with every operand of a tensor-core product rounded to BF16 where the kernels
    round it -- the standardised inputs x', the activations a1, a2 and the back-propagated
    pre-activation gradients d3, d2, d1 (each first as the FP32 value the kernels hold) -- and
    the bias gradients summed from the rounded d (the kernels append a column of ones to a layer's
    input).  rnd replaces the rounding (identity: the plain chain rule)."""
    r = bf16_round if rnd is None else rnd
    norm = np.asarray(norm, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(params)
    mx, isx = norm[:N_IN], norm[N_IN:2 * N_IN]
    a0 = r((np.asarray(X, dtype=np.float64) - mx) * isx)
    z1 = a0 @ W1.T + b1
    a1 = r(gelu(z1))
    z2 = a1 @ W2.T + b2
    a2 = r(gelu(z2))
    ys = a2 @ W3.T + b3
    n = len(ys)
    ts = (np.asarray(T, dtype=np.float64) - norm[2 * N_IN:2 * N_IN + N_OUT]) / norm[2 * N_IN + N_OUT:]
    e = ys - ts
    L = float(np.sum(e * e) / n)
    d3 = r(2.0 * e / n)
    d2 = r((d3 @ W3) * gelu_grad(z2))
    d1 = r((d2 @ W2) * gelu_grad(z1))
    g = np.concatenate([(d1.T @ a0).ravel(), d1.sum(axis=0), (d2.T @ a1).ravel(), d2.sum(axis=0),
                        (d3.T @ a2).ravel(), d3.sum(axis=0)])
    return L, g


def adam_step(w, m1, m2, grad, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) of FP64 arrays; returns (w, m1, m2)."""
    m1 = b1 * m1 + (1.0 - b1) * grad
    m2 = b2 * m2 + (1.0 - b2) * grad * grad
    mh = m1 / (1.0 - b1 ** t)
    vh = m2 / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m1, m2


def init_params(seed: int, scale: float = 1.0) -> np.ndarray:
    """He-style initial parameters from a seeded generator (biases zero), FP32 values."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((N_HIDDEN, N_IN)) * math.sqrt(2.0 / N_IN) * scale
    W2 = rng.standard_normal((N_HIDDEN, N_HIDDEN)) * math.sqrt(2.0 / N_HIDDEN) * scale
    W3 = rng.standard_normal((N_OUT, N_HIDDEN)) * math.sqrt(1.0 / N_HIDDEN) * scale
    z = np.zeros
    p = np.concatenate([W1.ravel(), z(N_HIDDEN), W2.ravel(), z(N_HIDDEN), W3.ravel(), z(N_OUT)])
    return p.astype(np.float32)
