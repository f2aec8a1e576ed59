"""Reference of the pair-selector network and its Adam optimiser (test
infrastructure only).

The network maps 8 normalised pair features through three hidden layers of
64 SiLU units to one output; the loss is the mean squared error.  Two forms:

* fp64: the plain definition in float64 (for finite-difference pins);
* bf16: float32 arithmetic with the inputs of every tensor-core product
  rounded to bfloat16 (round to nearest, ties to even) exactly where the GPU
  kernels round them -- the normalised features, the weights of layers 1-3,
  the hidden activations entering layers 2 and 3, and the gradients entering
  the backward products -- so the GPU can be compared with it closely.

Parameter layout (float32, 8977 values): W1[64][8], b1[64], W2[64][64],
b2[64], W3[64][64], b3[64], w4[64], b4, mean[8], scale[8].
"""
from __future__ import annotations

import numpy as np

H, F = 64, 8
NW = H * F + H + H * H + H + H * H + H + H + 1
NPARAMS = NW + 2 * F


def unpack(p):
    p = np.asarray(p)
    o = 0
    out = {}
    for name, shape in (("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)),
                        ("b3", (H,)), ("w4", (H,)), ("b4", (1,)), ("mean", (F,)), ("scale", (F,))):
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even); float32 out."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)


def silu(z):
    return z / (1 + np.exp(-z))


def silu_grad(z):
    s = 1 / (1 + np.exp(-z))
    return s * (1 + z * (1 - s))


def forward(params, feat, mode="bf16"):
    """Network outputs and the intermediate values [(z, h_in), ...]."""
    P = unpack(params)
    if mode == "fp64":
        dt = np.float64
        rnd = lambda v: v
    else:
        dt = np.float32
        rnd = bf16
    x = ((np.asarray(feat, dtype=dt) - P["mean"].astype(dt)) * P["scale"].astype(dt)).astype(dt)
    cache = []
    h = rnd(x)
    for W, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        z = (h.astype(np.float64) @ rnd(P[W].astype(dt)).astype(np.float64).T).astype(dt) + P[b].astype(dt)
        cache.append((z, h))
        a = silu(z).astype(dt)
        h = rnd(a) if W != "W3" else a
    y = (h.astype(np.float64) @ P["w4"].astype(np.float64)).astype(dt) + dt(P["b4"][0])
    return y, cache, h


def loss_and_grad(params, feat, label, mode="bf16"):
    """Mean squared error and its gradient with respect to the first NW
    parameters (the weights; the normalisation is fixed)."""
    P = unpack(params)
    dt = np.float64 if mode == "fp64" else np.float32
    rnd = (lambda v: v) if mode == "fp64" else bf16
    y, cache, h3 = forward(params, feat, mode)
    B = y.shape[0]
    r = y - np.asarray(label, dtype=dt)
    loss = float(np.mean(r.astype(np.float64) ** 2))
    dy = (2 * r / B).astype(dt)
    g = {}
    g["w4"] = (dy.astype(np.float64) @ h3.astype(np.float64)).astype(dt)
    g["b4"] = np.array([dy.astype(np.float64).sum()], dtype=dt)
    dz = (dy[:, None] * P["w4"][None, :].astype(dt)) * silu_grad(cache[2][0]).astype(dt)
    for L, (W, b) in reversed(list(enumerate((("W1", "b1"), ("W2", "b2"), ("W3", "b3"))))):
        z, hin = cache[L]
        g[W] = (dz.astype(np.float64).T @ hin.astype(np.float64)).astype(dt)
        g[b] = dz.astype(np.float64).sum(0).astype(dt)
        if L > 0:
            dh = (rnd(dz).astype(np.float64) @ rnd(P[W].astype(dt)).astype(np.float64)).astype(dt)
            dz = (dh * silu_grad(cache[L - 1][0])).astype(dt)
    flat = np.concatenate([g["W1"].ravel(), g["b1"], g["W2"].ravel(), g["b2"], g["W3"].ravel(), g["b3"],
                           g["w4"], g["b4"]])
    return loss, flat


def adam_step(params, m, v, grad, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) on the first NW
    parameters, in float64: the moment estimates decay by beta1 and beta2
    and take the gradient and its square, each estimate is divided by one
    minus its decay rate to the power of the step count (bias correction),
    and every weight moves by lr times the corrected first moment over
    (square root of the corrected second moment + eps).  The normalisation
    entries after the weights are left alone.  Returns new (params, m, v)."""
    p = np.array(params, dtype=np.float64)
    g = np.asarray(grad, dtype=np.float64)[:NW]
    m = beta1 * np.asarray(m, dtype=np.float64)[:NW] + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64)[:NW] + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    p[:NW] = p[:NW] - lr * m_hat / (np.sqrt(v_hat) + eps)
    return p, m, v
