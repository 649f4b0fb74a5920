"""FP64 reference of the surrogate network (test infrastructure only).

The surrogate maps five normalised drop parameters to two outputs: the
deformation D (regression) and a breakup logit (classification).  The network
is a plain multilayer perceptron: Linear(5, 128), then three Linear(128, 128),
each followed by SiLU, and a Linear(128, 2) head.  The training loss is
    L = mean((D_pred - D)^2) + mean(BCE(logit, breakup))
with BCE(z, y) = max(z, 0) - z y + log(1 + exp(-|z|)).  Adam with bias
correction updates FP32 master weights; the forward and backward passes use
the BF16-rounded copies of the weights, as the GPU kernels do.

Everything here is FP64 numpy, written from the definitions (no autograd);
the gradient pin in the tests checks it against central finite differences.
Only tests and the bench's CPU leg import this module.
"""
from __future__ import annotations

import numpy as np

WIDTHS = (5, 128, 128, 128, 128, 2)


def bf16_round(a):
    """Round float64 values to the nearest bfloat16 (round half to even)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    out = u.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def init_params(seed=0, widths=WIDTHS):
    """He-style initialisation: W ~ N(0, 2 / fan_in), b = 0.  Returns a list
    of (W [out, in], b [out]) in float64 (the FP32 master copy's values)."""
    rng = np.random.default_rng(seed)
    params = []
    for fin, fout in zip(widths[:-1], widths[1:]):
        W = rng.normal(0.0, np.sqrt(2.0 / fin), size=(fout, fin)).astype(np.float32).astype(np.float64)
        params.append([W, np.zeros(fout)])
    return params


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, X, round_weights=True):
    """Returns (outputs [n, 2], cache).  Weights are rounded to BF16 first
    when round_weights is set; biases stay FP32."""
    acts = [np.asarray(X, dtype=np.float64)]
    pre = []
    h = acts[0]
    last = len(params) - 1
    for k, (W, b) in enumerate(params):
        Wq = bf16_round(W) if round_weights else W
        z = h @ Wq.T + b
        pre.append(z)
        h = silu(z) if k < last else z
        acts.append(h)
    return h, (acts, pre)


def loss(out, yD, yB):
    """MSE on D plus binary cross-entropy on the logit, both averaged."""
    d = out[:, 0] - yD
    z = out[:, 1]
    bce = np.maximum(z, 0.0) - z * yB + np.log1p(np.exp(-np.abs(z)))
    return float(np.mean(d * d) + np.mean(bce))


def backward(params, cache, out, yD, yB, round_weights=True):
    """Gradients of loss() with respect to every W and b (same shapes)."""
    acts, pre = cache
    n = out.shape[0]
    g = np.zeros_like(out)
    g[:, 0] = 2.0 * (out[:, 0] - yD) / n
    g[:, 1] = (1.0 / (1.0 + np.exp(-out[:, 1])) - yB) / n
    grads = [None] * len(params)
    last = len(params) - 1
    for k in range(last, -1, -1):
        W, b = params[k]
        Wq = bf16_round(W) if round_weights else W
        if k < last:
            g = g * silu_grad(pre[k])
        grads[k] = [g.T @ acts[k], g.sum(axis=0)]
        g = g @ Wq
    return grads


def adam_step(params, grads, state, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update with bias correction; state is a list of (m, v) pairs
    matching params (created on first use)."""
    if not state:
        for W, b in params:
            state.append([np.zeros_like(W), np.zeros_like(W), np.zeros_like(b), np.zeros_like(b)])
    for (W, b), (gW, gb), st in zip(params, grads, state):
        for P, G, mi, vi in ((W, gW, 0, 1), (b, gb, 2, 3)):
            st[mi] = b1 * st[mi] + (1 - b1) * G
            st[vi] = b2 * st[vi] + (1 - b2) * G * G
            mh = st[mi] / (1 - b1 ** t)
            vh = st[vi] / (1 - b2 ** t)
            P -= lr * mh / (np.sqrt(vh) + eps)
    return state
