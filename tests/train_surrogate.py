"""Train the chemistry surrogate on FP64 oracle trajectories; write its weights.

    python tests/train_surrogate.py --out paper_1807_07094_gb300/data/surrogate_cosmic.npz

Data: free-running FP64 oracle runs (trace + sub-cycled chemistry, Sec. 2.4-2.8)
of lognormal cosmic fields at 64^3 with the cell size, density statistics and
source density of the 256^3 x 1000-source workload (16 sources, Ndot
log-uniform in [1e48, 1e51] ph/s, 1e5 K blackbody in 3 groups, H+He), one
seed per run, 20 steps each with dt = 0.02 Myr x 10^U(-0.5, 0.5) per step.
The runs advance with the paper's sub-cycling (eps = 0.1).  In every step a
seeded subset of cells is labelled with the converged solution of the same
rate equations: the oracle's update with every sub-step also capped at dt/200
and dt/400, Richardson-extrapolated (the scheme is first order in the step),
which agrees with a dt/3200 cap to ~5e-5.  (The paper's limiter bounds only
the hydrogen and energy changes per sub-step; its helium fractions carry a
first-order error of up to ~1e-2, so they are no label to learn.)  Each
labelled cell is one (state, rates, dt) -> (state') sample.

Training runs on the GPU through the package's trainer
(paper_1807_07094_gb300.train: BF16 tensor-core forward/backward, FP32
AdamW, features and raw targets from the library's own kernels, so that
training sees exactly what inference computes).  This script is test
infrastructure: it drives the oracle to make the labels, which the library
never does.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

DT0 = 0.02 * W.MYR


def converged(p, nH, x0, T0, g, h, dt):
    """Converged chemistry update: the oracle's sub-cycled update with every
    sub-step also capped at dt/200 and at dt/400, Richardson-extrapolated
    (the scheme is first order in the step)."""
    import oracle
    r = {}
    for m in (200, 400):
        r[m] = oracle.chem(p, nH, x0[0], x0[1], x0[2], T0, g, h, dt, min_sub=m)
        assert r[m][5] == 0
    x = [np.clip(2 * r[400][i] - r[200][i], 0.0, 1.0) for i in range(3)]
    T = np.maximum(2 * r[400][3] - r[200][3], 1.0)
    return x, T


def oracle_trajectory(args):
    """One free-running oracle run; returns per-step float32 sample arrays."""
    seed, n, nsrc, nsteps, per_step = args
    import oracle
    w = W.cosmic(n=n, nsrc=nsrc, seed=seed)
    p = w.params()
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    f32 = lambda a: np.asarray(a, np.float32).reshape(-1)
    xHI, xHeI, xHeII, T = (f32(a).astype(np.float64) for a in (w.xHI, w.xHeI, w.xHeII, w.T))
    nH = f32(w.nH)
    steps = []
    for k in range(nsteps):
        dt = float(DT0 * 10 ** rng.uniform(-0.5, 0.5))
        tr = oracle.trace(p, nH, xHI, xHeI, xHeII, w.src_pos, w.src_ndot)
        g = f32(tr["gamma"]).reshape(3, -1)
        h = f32(tr["heat"]).reshape(3, -1)
        x0 = np.stack([f32(xHI), f32(xHeI), f32(xHeII)])
        T0 = f32(T)
        # labels start from exactly the float32 inputs the network sees
        idx = np.sort(rng.choice(nH.size, min(per_step, nH.size), replace=False))
        xs, Ts = converged(p, nH[idx], x0[:, idx], T0[idx], g[:, idx], h[:, idx], dt)
        steps.append(dict(nH=nH[idx], x0=np.ascontiguousarray(x0[:, idx]), T0=T0[idx],
                          gamma=np.ascontiguousarray(g[:, idx]), heat=np.ascontiguousarray(h[:, idx]), dt=dt,
                          x1=np.stack([f32(v) for v in xs]), T1=f32(Ts)))
        # the run itself advances with the paper's sub-cycling
        xHI, xHeI, xHeII, T, _, capped = oracle.chem(p, nH, x0[0], x0[1], x0[2], T0, g, h, dt)
        assert capped == 0
    return seed, steps


def gather(seeds, n, nsrc, nsteps, per_step, workers):
    ctx = mp.get_context("spawn")
    jobs = [(s, n, nsrc, nsteps, per_step) for s in seeds]
    out = {}
    with ctx.Pool(min(workers, len(jobs))) as pool:
        for seed, steps in pool.imap_unordered(oracle_trajectory, jobs):
            out[seed] = steps
            print(f"  oracle seed {seed}: {len(steps)} steps", flush=True)
    return [st for s in seeds for st in out[s]]


def _label_chunk(args):
    """Converged update of one chunk of sampled cells (a spawned worker)."""
    p, nH, x0, T0, g, h, dt = args
    xs, Ts = converged(p, nH.astype(np.float64), x0.astype(np.float64), T0.astype(np.float64),
                       g.astype(np.float64), h.astype(np.float64), dt)
    return np.stack([np.asarray(v, np.float32) for v in xs]), np.asarray(Ts, np.float32)


def gpu_states(configs, nsteps, per_step, workers, seed0=7919):
    """Cell samples of the C4 configurations: cosmic fields at 128^3 and 256^3
    with the benchmark's cell size, density statistics and source density,
    advanced on the GPU (trace + the paper's sub-cycled chemistry, both matched
    to the oracle by the parity tests) with dt = 0.02 Myr x 10^U(-0.5, 0.5) per
    step; each step samples per_step cells, half uniformly and half among the
    cells the radiation reaches (Gamma_HI dt > 1e-4), and the oracle labels
    them with its converged update in spawned worker processes.  configs:
    (n, nsrc, seed) triples."""
    import torch
    import paper_1807_07094_gb300 as P
    steps = []
    pool = mp.get_context("spawn").Pool(workers)
    pending = []
    for (n, nsrc, seed) in configs:
        w = W.cosmic(n=n, nsrc=nsrc, seed=seed)
        p = w.params()
        rng = np.random.Generator(np.random.PCG64(seed + seed0))
        nH = np.asarray(w.nH, np.float32).reshape(-1)
        with P.Arc(w.n, w.box_cm, p) as a:
            a.set_fields(w.nH, w.xHI, w.xHeI, w.xHeII, w.T)
            a.add_sources(w.src_pos, w.src_ndot)
            for k in range(nsteps):
                dt = float(DT0 * 10 ** rng.uniform(-0.5, 0.5))
                g, h, _ = a.trace(dt, budget=True)          # budget=True waits for the rates
                g = g.cpu().numpy().reshape(3, -1)
                h = h.cpu().numpy().reshape(3, -1)
                xs = [np.asarray(v, np.float32).reshape(-1) for v in a.get_fields()]
                lit = np.flatnonzero(g[0] * dt > 1e-4)
                half = per_step // 2
                idx = rng.choice(nH.size, per_step - min(half, lit.size), replace=False)
                if lit.size:
                    idx = np.concatenate([idx, rng.choice(lit, min(half, lit.size), replace=False)])
                idx = np.unique(idx)
                st = dict(nH=nH[idx], x0=np.stack([xs[q][idx] for q in range(3)]), T0=xs[3][idx],
                          gamma=np.ascontiguousarray(g[:, idx]), heat=np.ascontiguousarray(h[:, idx]), dt=dt)
                chunks = np.array_split(np.arange(idx.size), max(1, idx.size // 2048))
                pending.append((st, [pool.apply_async(_label_chunk, ((p, st["nH"][c], st["x0"][:, c], st["T0"][c],
                                                                      st["gamma"][:, c], st["heat"][:, c], dt),))
                                     for c in chunks]))
                a.chem(dt)
        print(f"  gpu states n={n} seed={seed}: {nsteps} steps", flush=True)
    for st, res in pending:
        out = [r.get() for r in res]
        st["x1"] = np.concatenate([o[0] for o in out], axis=1)
        st["T1"] = np.concatenate([o[1] for o in out])
        steps.append(st)
    pool.close()
    pool.join()
    return steps


def evaluate(path_new, path_old=None, n=256, nsrc=1000, seed=1807, nsteps=3):
    """Surrogate on a held-out state (the 256^3 benchmark field after nsteps):
    accepted fraction with the new weights, the old ones and the predictor
    alone (zero network output), and the accepted cells' distance from the
    oracle's converged update on a seeded probe."""
    import torch
    import paper_1807_07094_gb300 as P
    w = W.cosmic(n=n, nsrc=nsrc, seed=seed)
    p = w.params()
    res = {}
    with P.Arc(w.n, w.box_cm, p) as a:
        a.set_fields(w.nH, w.xHI, w.xHeI, w.xHeII, w.T)
        a.add_sources(w.src_pos, w.src_ndot)
        for _ in range(nsteps):
            a.step(w.dt_s)
        state = a.get_fields()
        g, h, _ = a.trace(w.dt_s, budget=True)
        g = g.cpu().numpy().reshape(3, -1)
        h = h.cpu().numpy().reshape(3, -1)
        n3 = w.n ** 3
        rng = np.random.Generator(np.random.PCG64(99))
        lit = np.flatnonzero(g[0] * w.dt_s > 1e-4)
        probe = np.unique(np.concatenate([rng.choice(n3, 2048, replace=False), rng.choice(lit, 2048, replace=False)]))
        f = lambda v: np.asarray(v, np.float32).reshape(-1)[probe]
        xs, Ts = converged(p, f(w.nH).astype(np.float64), np.stack([f(state[q]) for q in range(3)]).astype(np.float64),
                           f(state[3]).astype(np.float64), g[:, probe].astype(np.float64),
                           h[:, probe].astype(np.float64), w.dt_s)
        arms = {"new": P.load_surrogate(path_new)[:2]}
        if path_old:
            arms["old"] = P.load_surrogate(path_old)[:2]
        pn, nn = arms["new"]
        n0 = nn.copy()
        n0[24:28] = 0.0
        arms["predictor"] = (np.zeros_like(pn), n0)
        for name, (prm, nrm) in arms.items():
            a.set_fields(w.nH, *state)
            a.set_surrogate(None)
            a.chem(w.dt_s)
            plain = [f(v) for v in a.get_fields()]
            a.set_fields(w.nH, *state)
            a.set_surrogate(prm, nrm)
            a.chem(w.dt_s)
            st = a.stats()
            out = [f(v) for v in a.get_fields()]
            a.set_surrogate(None)
            acc = np.zeros(probe.size, bool)
            for u, v in zip(plain, out):
                acc |= u != v
            dx = max(float(np.abs(out[q] - xs[q])[acc].max(initial=0.0)) for q in range(3))
            dT = float(np.abs(out[3] / Ts - 1)[acc].max(initial=0.0))
            res[name] = dict(accepted_frac=st["surrogate_cells"] / n3, chem_ms=st["chem_ms"],
                             probe_accepted=int(acc.sum()), probe_max_dx=dx, probe_max_dT_rel=dT)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--seeds", default="101,102,103,104,105,106,107,108")
    ap.add_argument("--per-step", type=int, default=16384, help="labelled cells per step")
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--nsrc", type=int, default=16)
    ap.add_argument("--nsteps", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--wd", type=float, default=1e-5)
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--states", default="oracle", choices=["oracle", "gpu"],
                    help="oracle: free-running oracle runs at --n; gpu: the C4 configurations (128^3 and "
                         "256^3 cosmic fields) advanced on the GPU, cells labelled by the oracle")
    ap.add_argument("--configs", default="128:125:201,128:125:202,128:125:203,128:125:204,256:1000:301,256:1000:302",
                    help="n:nsrc:seed triples for --states gpu")
    ap.add_argument("--evaluate-against", default="", help="old weights file to compare on the held-out state")
    a = ap.parse_args()
    seeds = [int(s) for s in a.seeds.split(",")]
    t0 = time.time()
    if a.states == "gpu":
        configs = [tuple(int(v) for v in c.split(":")) for c in a.configs.split(",")]
        steps = gpu_states(configs, a.nsteps, a.per_step, a.workers)
        seeds = [c[2] for c in configs]
    else:
        steps = gather(seeds, a.n, a.nsrc, a.nsteps, a.per_step, a.workers)
    t1 = time.time()
    print(f"oracle data: {len(steps)} steps in {t1 - t0:.0f} s", flush=True)
    from paper_1807_07094_gb300 import train as T
    P, norm, hist, nsamples = T.train_surrogate(steps, W.cosmic(n=8, nsrc=1).params(), a.epochs, a.batch,
                                                a.lr, a.wd, seeds[0])
    t2 = time.time()
    recipe = ("FP64 oracle trajectories of lognormal cosmic fields (sigma_ln 1.5, P(k)~k^-3, mean nH 2e-4)"
              if a.states == "oracle" else
              "cosmic fields " + a.configs + " (n:nsrc:seed; sigma_ln 1.5, P(k)~k^-3, mean nH 2e-4) advanced on the "
              "GPU, half of each step's cells sampled where Gamma_HI dt > 1e-4")
    meta = dict(recipe=recipe + "; labels: the oracle's converged update (Richardson of sub-step caps dt/200, dt/400)",
                nsteps=a.nsteps, seeds=seeds, per_step=a.per_step, samples=nsamples,
                epochs=a.epochs,
                batch=a.batch, lr=a.lr, wd=a.wd, loss=hist, oracle_s=round(t1 - t0, 1), train_s=round(t2 - t1, 1))
    if a.states == "oracle":
        meta.update(n=a.n, nsrc=a.nsrc)
    T.save_weights(a.out, P, norm, meta)
    print(json.dumps(meta))
    if a.evaluate_against is not None and a.states == "gpu":
        print("EVAL " + json.dumps(evaluate(a.out, a.evaluate_against or None)), flush=True)


if __name__ == "__main__":
    main()
