"""FP64 reference of the chemistry surrogate's network (test infrastructure).

A plain NumPy statement of the MLP the library runs on the tensor cores:
12 -> 64 -> 64 -> 64 -> 4, SiLU between layers, mean-squared error over the 4
normalised outputs, and its gradient by backpropagation.  With ``bf16=True``
the forward pass rounds what the device rounds to bfloat16 (weights, hidden
activations; the output gradient and the hidden-layer gradients in the
backward pass; the FP32 normalised inputs enter as the sum of two bfloat16
halves, hi = bf16(v) and lo = bf16(v - hi)) and keeps everything else in
FP64, so that the device's FP32 accumulation is the only remaining difference.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 12, 64, 4
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_H, N_H)), ("b3", (N_H,)), ("W4", (N_OUT, N_H)), ("b4", (N_OUT,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
NNORM = 2 * N_IN + 3 * N_OUT


def unpack(P):
    P = np.asarray(P, np.float64)
    assert P.size == NPARAMS
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = P[o:o + k].reshape(shp)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(seed: int):
    """Seeded He-style initialisation (biases zero)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = {}
    for name, shp in SHAPES:
        if name[0] == "W":
            d[name] = rng.normal(0.0, np.sqrt(2.0 / shp[1]), shp)
        else:
            d[name] = np.zeros(shp)
    return pack(d).astype(np.float32)


def split_norm(norm):
    q = np.asarray(norm, np.float64)
    assert q.size == NNORM
    return dict(in_mu=q[:N_IN], in_sd=q[N_IN:2 * N_IN], out_mu=q[2 * N_IN:2 * N_IN + N_OUT],
                out_sd=q[2 * N_IN + N_OUT:2 * N_IN + 2 * N_OUT], out_s=q[2 * N_IN + 2 * N_OUT:])


def split_bf16(v):
    """FP32 values as the sum of their bfloat16 hi and lo halves (float64)."""
    v32 = np.asarray(v, np.float32)
    hi = bf16(v32)
    lo = bf16(v32 - hi.astype(np.float32))
    return hi + lo


def normalise_inputs(X, norm, fp32: bool = False):
    """(x - mu) / sd; with fp32 in FP32 arithmetic as the device forms it."""
    q = split_norm(norm)
    if fp32:
        X32 = np.asarray(X, np.float32)
        return (X32 - q["in_mu"].astype(np.float32)) / q["in_sd"].astype(np.float32)
    return (np.asarray(X, np.float64) - q["in_mu"]) / q["in_sd"]


def targets_to_output(R, norm):
    """Step changes r -> normalised network targets (asinh(r / s) - mu) / sd."""
    q = split_norm(norm)
    return (np.arcsinh(np.asarray(R, np.float64) / q["out_s"]) - q["out_mu"]) / q["out_sd"]


def output_to_change(O, norm):
    q = split_norm(norm)
    return q["out_s"] * np.sinh(np.asarray(O, np.float64) * q["out_sd"] + q["out_mu"])


def forward(P, Xn, bf16_round: bool = False):
    """Normalised inputs Xn [n, 12] -> normalised outputs [n, 4] and the cache."""
    p = unpack(P)
    rnd = bf16 if bf16_round else (lambda a: np.asarray(a, np.float64))
    A = split_bf16(Xn) if bf16_round else np.asarray(Xn, np.float64)
    cache = [A]
    Zs = []
    for l in (1, 2, 3):
        Z = A @ rnd(p[f"W{l}"]).T + p[f"b{l}"]
        A = rnd(silu(Z))
        Zs.append(Z)
        cache.append(A)
    out = A @ rnd(p["W4"]).T + p["b4"]
    return out, (cache, Zs)


def loss_grad(P, Xn, Yn, bf16_round: bool = False):
    """Mean-squared error over samples and outputs, and its gradient [NPARAMS]."""
    p = unpack(P)
    rnd = bf16 if bf16_round else (lambda a: np.asarray(a, np.float64))
    out, (acts, Zs) = forward(P, Xn, bf16_round)
    n = out.shape[0]
    diff = out - np.asarray(Yn, np.float64)
    loss = float(np.sum(diff * diff) / (N_OUT * n))
    g = {}
    dY = 2.0 * diff / (N_OUT * n)
    g["b4"] = dY.sum(axis=0)
    dYr = rnd(dY)
    g["W4"] = dYr.T @ acts[3]
    dA = dYr @ rnd(p["W4"])
    for l in (3, 2, 1):
        dZ = dA * dsilu(Zs[l - 1])
        g[f"b{l}"] = dZ.sum(axis=0)
        dZr = rnd(dZ)
        g[f"W{l}"] = dZr.T @ acts[l - 1]
        dA = dZr @ rnd(p[f"W{l}"])
    return loss, pack(g)
