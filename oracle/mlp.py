"""CPU oracle of the warm-start MLP (no counterpart in the paper).

The paper starts every Newton solve from the previous velocity (Algorithm 3,
v <- v_n).  The learned warm start replaces that start by
v0 = b + s_out r_I MLP(features) on free nodes (0 on clamped nodes), where b
is the polynomial extrapolation of the velocity history that is available
(cubic from v_n .. v_{n-3}; quadratic, linear or v_n itself when fewer
previous velocities exist): the network learns a correction of it.  Inputs
per node: the first, second and third backward differences of the velocity
history, each divided by its own scale, the nine divided by their norm r_I
(so the map does not depend on the amplitude of the motion), and the fixed
flag.
Per-node MLP 10 -> 64 -> 64 -> 64 -> 3, tanh hidden layers, linear output.
Weights and activations are bfloat16, products are accumulated in float32.

This module restates the forward pass, the mean-squared-error loss and the
backward pass with plain numpy.  `bf16=True` rounds weights and stored
activations to bfloat16 (round to nearest even) exactly where the CUDA kernels
do; `bf16=False, dtype=float64` is the smooth reference that finite
differences pin.

Parameter vector layout (length 9219): W1 (64x10), b1 (64), W2 (64x64), b2 (64),
W3 (64x64), b3 (64), W4 (3x64), b4 (3); W rows are outputs.
"""
from __future__ import annotations

import numpy as np

SIZES = [(64, 10), (64,), (64, 64), (64,), (64, 64), (64,), (3, 64), (3,)]
NPARAM = sum(int(np.prod(s)) for s in SIZES)


def unpack(theta):
    out, o = [], 0
    for s in SIZES:
        n = int(np.prod(s))
        out.append(theta[o:o + n].reshape(s))
        o += n
    return out


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    x = np.asarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    r = np.where(np.isnan(x), b, r)
    return r.astype(np.uint32).view(np.float32)


def init_params(rng):
    """Glorot-uniform weights, zero biases (float32)."""
    theta = []
    for s in SIZES:
        if len(s) == 2:
            lim = np.sqrt(6.0 / (s[0] + s[1]))
            theta.append(rng.uniform(-lim, lim, size=s).astype(np.float32).ravel())
        else:
            theta.append(np.zeros(s, np.float32))
    return np.concatenate(theta)


def forward(theta, x, bf16=True, dtype=np.float32):
    """Returns (out, cache).  x: (N, 10)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = [a.astype(dtype) for a in unpack(theta)]
    rnd = bf16_round if bf16 else (lambda a: a)
    if bf16:
        W1, W2, W3, W4 = rnd(W1), rnd(W2), rnd(W3), rnd(W4)
        b1, b2, b3, b4 = rnd(b1), rnd(b2), rnd(b3), rnd(b4)
    x = rnd(np.asarray(x, dtype=dtype))
    h1 = rnd(np.tanh(x @ W1.T + b1))
    h2 = rnd(np.tanh(h1 @ W2.T + b2))
    h3 = rnd(np.tanh(h2 @ W3.T + b3))
    out = h3 @ W4.T + b4
    return out, (x, h1, h2, h3, (W1, W2, W3, W4))


def mse(out, target, weight):
    """L = sum_n w_n ||out_n - target_n||^2 and dL/dout."""
    d = out - target
    return float(np.sum(weight[:, None] * d * d)), 2.0 * weight[:, None] * d


def backward(theta, cache, dout):
    """Gradient of sum(dout * out) with respect to theta (same layout)."""
    x, h1, h2, h3, (W1, W2, W3, W4) = cache
    g4 = dout.T @ h3
    gb4 = dout.sum(0)
    d3 = (dout @ W4) * (1.0 - h3 * h3)
    g3 = d3.T @ h2
    gb3 = d3.sum(0)
    d2 = (d3 @ W3) * (1.0 - h2 * h2)
    g2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (1.0 - h1 * h1)
    g1 = d1.T @ x
    gb1 = d1.sum(0)
    return np.concatenate([a.ravel() for a in (g1, gb1, g2, gb2, g3, gb3, g4, gb4)])


def adam_step(theta, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update on the float32 master parameters (in place)."""
    m[:] = b1 * m + (1 - b1) * grad
    v[:] = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    theta -= lr * mh / (np.sqrt(vh) + eps)
    return theta


def backward_differences(v_n, v_prev=None, v_prev2=None, v_prev3=None):
    """First, second and third backward differences of the velocity history at
    step n (nabla v_n = v_n - v_{n-1}, nabla^2 v_n = v_n - 2 v_{n-1} + v_{n-2},
    nabla^3 v_n = v_n - 3 v_{n-1} + 3 v_{n-2} - v_{n-3}); a difference that
    needs a missing velocity is zero.  Each (nn, 3)."""
    v = [np.asarray(a, dtype=np.float64).reshape(-1, 3) if a is not None else None
         for a in (v_n, v_prev, v_prev2, v_prev3)]
    z = np.zeros_like(v[0])
    d1 = v[0] - v[1] if v[1] is not None else z
    d2 = v[0] - 2.0 * v[1] + v[2] if v[1] is not None and v[2] is not None else z
    d3 = (v[0] - 3.0 * v[1] + 3.0 * v[2] - v[3]
          if v[1] is not None and v[2] is not None and v[3] is not None else z)
    return d1, d2, d3


def extrapolation(v_n, v_prev=None, v_prev2=None, v_prev3=None):
    """Polynomial extrapolation of the velocity history to step n + 1 (Newton's
    backward-difference form): v_n + nabla v_n + nabla^2 v_n + nabla^3 v_n, the
    terms that need a missing velocity dropped (cubic, quadratic, linear or
    v_n itself)."""
    d1, d2, d3 = backward_differences(v_n, v_prev, v_prev2, v_prev3)
    return np.asarray(v_n, dtype=np.float64).reshape(-1, 3) + d1 + d2 + d3


def node_scale(v_n, v_prev, v_prev2, v_prev3, s1, s2, s3):
    """r_I = || (nabla v / s1, nabla^2 v / s2, nabla^3 v / s3) || per node (the
    9 scaled differences of node I): the network sees the history divided by
    it and its correction is multiplied by it, so the learned map does not
    depend on the amplitude of the motion (the extrapolation error is a
    degree-one homogeneous function of the history)."""
    d1, d2, d3 = backward_differences(v_n, v_prev, v_prev2, v_prev3)
    return np.sqrt(np.sum((d1 / s1) ** 2 + (d2 / s2) ** 2 + (d3 / s3) ** 2, axis=1))


def features(v_n, v_prev, v_prev2, v_prev3, fixed_mask, s1, s2, s3):
    """Per-node inputs: (nabla v / s1, nabla^2 v / s2, nabla^3 v / s3) / r_I
    (three columns each; zero where r_I = 0) and the fixed flag."""
    d1, d2, d3 = backward_differences(v_n, v_prev, v_prev2, v_prev3)
    r = node_scale(v_n, v_prev, v_prev2, v_prev3, s1, s2, s3)
    inv = np.where(r > 0.0, 1.0 / np.where(r > 0.0, r, 1.0), 0.0)[:, None]
    return np.concatenate([d1 / s1 * inv, d2 / s2 * inv, d3 / s3 * inv,
                           np.asarray(fixed_mask, np.float64)[:, None]], axis=1)


def target(v_next, v_n, v_prev, v_prev2, v_prev3, fixed_mask, s1, s2, s3, s_out):
    """Training target: (v_{n+1} - extrapolation) / (s_out r_I), zero on fixed
    nodes and where r_I = 0."""
    r = node_scale(v_n, v_prev, v_prev2, v_prev3, s1, s2, s3)
    e = np.asarray(v_next, dtype=np.float64).reshape(-1, 3) - extrapolation(v_n, v_prev, v_prev2, v_prev3)
    t = np.where(r[:, None] > 0.0, e / (s_out * np.where(r > 0.0, r, 1.0))[:, None], 0.0)
    t[np.asarray(fixed_mask, bool)] = 0.0
    return t


def start_velocity(out, v_n, v_prev, v_prev2, v_prev3, fixed_mask, s1, s2, s3, s_out):
    """v0 = extrapolation + s_out r_I out on free nodes, 0 on fixed nodes (out
    may be None: the extrapolation alone)."""
    v0 = extrapolation(v_n, v_prev, v_prev2, v_prev3)
    if out is not None:
        r = node_scale(v_n, v_prev, v_prev2, v_prev3, s1, s2, s3)
        v0 = v0 + s_out * r[:, None] * np.asarray(out, dtype=np.float64).reshape(-1, 3)
    v0[np.asarray(fixed_mask, bool)] = 0.0
    return v0
