"""Training of the chemistry surrogate on the GPU (the learned part's trainer).

Given labelled cells -- start state, rates, time step and the chemistry
update to learn -- this module forms the network's features and raw targets
with the library's own feature and target kernels (so training sees exactly
what inference computes), fits the normalisation, and trains the 12 -> 64 ->
64 -> 64 -> 4 SiLU network with the library's BF16 tensor-core forward and
backward passes and FP32 AdamW (arc_mlp_train_step).  It writes the weights
file the chemistry kernel loads (load_surrogate).

Where the labels come from is the caller's business: the project's data
script (tests/train_surrogate.py) labels cells with the FP64 oracle's
converged update; this module never runs the oracle.
"""
from __future__ import annotations

import json
import os
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import arc

N_IN, N_H, N_OUT = 12, 64, 4
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_H, N_H)), ("b3", (N_H,)), ("W4", (N_OUT, N_H)), ("b4", (N_OUT,))]
# asinh scales of the 4 raw targets (corrections of x_HI, x_HeI, x_HeII, log10 T)
OUT_S = np.array([1e-6, 1e-6, 1e-6, 1e-5])


def init_params(seed: int) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, in the flat
    parameter order of the library (W1, b1, W2, b2, W3, b3, W4, b4)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for name, shp in SHAPES:
        if name[0] == "W":
            parts.append(rng.normal(0.0, np.sqrt(2.0 / shp[1]), shp).reshape(-1))
        else:
            parts.append(np.zeros(int(np.prod(shp))))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == arc.MLP_NPARAMS
    return p


def device_samples(steps: Sequence[Dict], params: dict, stream: Optional[int] = None):
    """Features X [N, 12] and raw targets R [N, 4] (corrections of the physics
    predictor) on the GPU, by the library's kernels, for labelled cells.

    Each element of ``steps`` holds float32 arrays nH [m], x0 [3, m] (x_HI,
    x_HeI, x_HeII), T0 [m], gamma [3, m], heat [3, m], the labels x1 [3, m],
    T1 [m] and the time step dt [s]; ``params`` are the workload parameters
    (helium fraction, rate options) the labels were made with."""
    import torch
    dev = torch.device("cuda")
    Xs, Rs = [], []
    with arc.Arc(8, 1e21, params, stream=stream) as ctx:
        for st in steps:
            t = {k: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).to(dev)
                 for k, v in st.items() if k != "dt"}
            m = t["nH"].numel()
            X = torch.empty((m, N_IN), dtype=torch.float32, device=dev)
            R = torch.empty((m, N_OUT), dtype=torch.float32, device=dev)
            torch.cuda.synchronize()
            arc.arc_mlp_features(t["nH"], t["x0"][0], t["x0"][1], t["x0"][2], t["T0"], t["gamma"],
                                 t["heat"], st["dt"], X, stream)
            ctx.mlp_targets(t["nH"], t["x0"], t["T0"], t["gamma"], t["heat"], t["x1"], t["T1"], st["dt"], R)
            torch.cuda.synchronize()
            Xs.append(X)
            Rs.append(R)
    return torch.cat(Xs), torch.cat(Rs)


def fit_norm(X, R) -> np.ndarray:
    """Normalisation block (36 floats): input mean and spread, mean and spread
    of the asinh-scaled targets, and the asinh scales."""
    import torch
    in_mu = X.double().mean(0)
    in_sd = X.double().std(0).clamp_min(1e-3)
    s = torch.tensor(OUT_S, dtype=torch.float64, device=R.device)
    U = torch.asinh(R.double() / s)
    out_mu = U.mean(0)
    out_sd = U.std(0).clamp_min(1e-3)
    norm = torch.cat([in_mu, in_sd, out_mu, out_sd, s])
    return norm.float().cpu().numpy()


def normalise(X, R, norm):
    import torch
    q = torch.from_numpy(np.asarray(norm, np.float64)).to(X.device)
    Xn = ((X.double() - q[:N_IN]) / q[N_IN:2 * N_IN]).float()
    Yn = ((torch.asinh(R.double() / q[32:36]) - q[24:28]) / q[28:32]).float()
    return Xn.contiguous(), Yn.contiguous()


def train(Xn, Yn, epochs: int, batch: int, lr0: float, wd: float, seed: int, stream: Optional[int] = None,
          log: Callable[[str], None] = print) -> Tuple[np.ndarray, List[float]]:
    """AdamW on the mean-squared error of the normalised targets, cosine
    learning-rate schedule, every step on the library's trainer."""
    import torch
    N = Xn.shape[0] // batch * batch
    tr = arc.MlpTrainer(batch, stream)
    tr.set_params(init_params(seed))
    g = torch.Generator(device="cpu").manual_seed(seed)
    nb = N // batch
    total = max(1, epochs * nb)
    k = 0
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(Xn.shape[0], generator=g)[:N].to(Xn.device)
        Xp, Yp = Xn[perm].contiguous(), Yn[perm].contiguous()
        acc = 0.0
        for b in range(nb):
            lr = lr0 * 0.5 * (1 + np.cos(np.pi * k / total)) + 1e-6
            want = b % 50 == 0
            loss = tr.step(Xp[b * batch:(b + 1) * batch], Yp[b * batch:(b + 1) * batch], batch, lr, wd, want)
            if want:
                acc = loss if acc == 0.0 else 0.8 * acc + 0.2 * loss
            k += 1
        hist.append(acc)
        log(f"  epoch {ep}: loss {acc:.3e}")
    P = tr.get_params()
    tr.close()
    return P, hist


def save_weights(path: str, params: np.ndarray, norm: np.ndarray, meta: dict) -> None:
    """The weights file load_surrogate reads: parameters, normalisation, and a
    JSON description of how they were made."""
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.savez(path, params=np.asarray(params, np.float32), norm=np.asarray(norm, np.float32),
             meta=json.dumps(meta))


def train_surrogate(steps: Sequence[Dict], workload_params: dict, epochs: int = 60, batch: int = 4096,
                    lr: float = 2e-3, wd: float = 1e-5, seed: int = 101, log: Callable[[str], None] = print):
    """Labelled cells -> (parameters, normalisation, loss history, sample count),
    all on the GPU on a stream of its own."""
    import torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        X, R = device_samples(steps, workload_params, s.cuda_stream)
        s.synchronize()
        norm = fit_norm(X, R)
        Xn, Yn = normalise(X, R, norm)
        s.synchronize()
        P, hist = train(Xn, Yn, epochs, batch, lr, wd, seed, s.cuda_stream, log)
    return P, norm, hist, int(X.shape[0])
