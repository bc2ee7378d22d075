"""GPU chemistry / energy update (libarc through the C ABI) against the FP64 oracle.

Bars: neutral fractions within 1e-4 absolute of the oracle after every update
and after free-running runs; temperature within 1e-3 relative.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1807_07094_gb300 as P
import workloads as W
from helpers import gpu_trace, oracle_trace

pytestmark = pytest.mark.gpu

X_ATOL = 1e-4
T_RTOL = 1e-3


def gpu_chem_cells(params, nH, xHI, xHeI, xHeII, T, gamma, heat, dt):
    """Run arc_chem_update on a flat set of cells laid out as an n^3 grid
    (padded with empty cells)."""
    ncell = nH.size
    n = int(np.ceil(ncell ** (1 / 3)))
    pad = n ** 3 - ncell
    f = lambda a: np.concatenate([np.asarray(a, np.float32).ravel(), np.zeros(pad, np.float32)])
    ft = lambda a: np.concatenate([np.asarray(a, np.float32).ravel(), np.ones(pad, np.float32) * 100])
    with P.Arc(n, 1e21 * n, params) as a:
        a.set_fields(f(nH).reshape(n, n, n), f(xHI).reshape(n, n, n), f(xHeI).reshape(n, n, n),
                     f(xHeII).reshape(n, n, n), ft(T).reshape(n, n, n))
        # rates go straight into the context's rate buffers
        g, h, _ = a.trace(1.0, budget=False)
        torch.cuda.synchronize()   # the trace runs on the context's own stream
        gg = torch.from_numpy(np.stack([f(gamma[s]) for s in range(3)]).reshape(3, n, n, n)).cuda()
        hh = torch.from_numpy(np.stack([f(heat[s]) for s in range(3)]).reshape(3, n, n, n)).cuda()
        g.copy_(gg)
        h.copy_(hh)
        torch.cuda.synchronize()
        a.chem(dt)
        out = a.get_fields()
        st = a.stats()
    return [o.ravel()[:ncell] for o in out], st


@pytest.mark.parametrize("seed", [0, 1])
def test_chem_random_cells(seed):
    m = 4096
    nH, xHI, xHeI, xHeII, T = W.random_gas(m, seed)
    gamma, heat = W.random_rates(m, seed, gmax=1e-12)
    p = W.thermal_128().params()
    dt = 0.02 * W.MYR
    (gx, gxe1, gxe2, gT), st = gpu_chem_cells(p, nH, xHI, xHeI, xHeII, T, gamma, heat, dt)
    ox, oxe1, oxe2, oT, nsub, capped = oracle.chem(p, nH, xHI, xHeI, xHeII, T, gamma, heat, dt)
    assert capped == 0 and st["chem_capped"] == 0
    assert np.max(np.abs(gx - ox)) < X_ATOL
    assert np.max(np.abs(gxe1 - oxe1)) < X_ATOL
    assert np.max(np.abs(gxe2 - oxe2)) < X_ATOL
    assert np.max(np.abs(gT / oT - 1)) < T_RTOL
    assert st["chem_fp64_substeps"] > 0       # the x_HI < 1e-4 branch was exercised


def test_chem_isothermal_fixed_alpha():
    m = 2000
    nH, xHI, _, _, T = W.random_gas(m, 5, Y=0.0)
    T[:] = 1e4
    gamma, heat = W.random_rates(m, 5, gmax=1e-11)
    p = W.stromgren_32().params()
    z = np.zeros(m, np.float32)
    (gx, _, _, gT), st = gpu_chem_cells(p, nH, xHI, z, z, T, gamma, heat, 1.0 * W.MYR)
    ox, _, _, oT, nsub, capped = oracle.chem(p, nH, xHI, z, z, T, gamma, heat, 1.0 * W.MYR)
    assert np.max(np.abs(gx - ox)) < X_ATOL
    assert np.all(gT == 1e4)


def free_run_gpu(w, nsteps, use_graph):
    with P.Arc(w.n, w.box_cm, w.params()) as a:
        a.set_fields(w.nH, w.xHI, w.xHeI, w.xHeII, w.T)
        a.add_sources(w.src_pos, w.src_ndot)
        for k in range(nsteps):
            if use_graph:
                a.step(w.dt_s)
            else:
                a.trace(w.dt_s, budget=False)
                a.chem(w.dt_s)
        return a.get_fields()


@pytest.mark.parametrize("use_graph", [False, True])
def test_free_running_stromgren(use_graph):
    """C1 run (32^3, 50 x 1 Myr): x after the run within 1e-4 of the oracle's."""
    w = W.stromgren_32()
    gx, _, _, _ = free_run_gpu(w, w.nsteps, use_graph)
    ox, _, _, _, _ = oracle.run(w.params(), w, w.nsteps)
    err = np.abs(gx - ox)
    assert err.max() < X_ATOL, (err.max(), np.unravel_index(err.argmax(), err.shape))


def test_free_running_thermal_short():
    """H+He with heating/cooling (128^3 setup at 40^3), 10 steps of 0.5 Myr."""
    w = W.thermal_128(n=40, box_kpc=6.6 * 40 / 128)
    gx, gxe1, gxe2, gT = free_run_gpu(w, 10, True)
    ox, oxe1, oxe2, oT, _ = oracle.run(w.params(), w, 10)
    assert np.abs(gx - ox).max() < X_ATOL
    assert np.abs(gxe1 - oxe1).max() < X_ATOL
    assert np.abs(gxe2 - oxe2).max() < X_ATOL
    assert np.abs(gT / oT - 1).max() < T_RTOL


def test_graph_step_matches_eager():
    w = W.cosmic(n=48, nsrc=8, seed=21)
    a = free_run_gpu(w, 3, False)
    b = free_run_gpu(w, 3, True)
    # the cell sums are FP32 atomics, so two runs differ by the order of the
    # additions (~1e-7 relative per cell).  Three chemistry steps carry that to
    # a few 1e-6 in the ionised fractions; a cell that the front is crossing
    # heats from ~1e2 K to ~1e4 K within the step, so its temperature moves by
    # far more than its rates and is held per cell to the rates' own bar.
    for x, y in zip(a[:3], b[:3]):
        assert np.abs(x - y).max() <= 1e-5
    Ta, Tb = a[3].astype(np.float64), b[3].astype(np.float64)
    rel = np.abs(Ta - Tb) / Ta
    assert rel.max() <= 1e-4, (rel.max(), np.unravel_index(rel.argmax(), rel.shape))


def test_rt_timestep_matches_oracle():
    """Sec. 2.9 time-step minima on random gas and rates: the GPU reduction
    against the oracle's loop over the same cells."""
    n = 16
    m = n ** 3
    nH, xHI, xHeI, xHeII, T = W.random_gas(m, 7)
    gamma, heat = W.random_rates(m, 7, gmax=1e-12)
    p = dict(W.thermal_128().params(), n=n, box_cm=1e21 * n)
    sh = (n, n, n)
    with P.Arc(n, 1e21 * n, p) as a:
        a.set_fields(nH.reshape(sh), xHI.reshape(sh), xHeI.reshape(sh), xHeII.reshape(sh), T.reshape(sh))
        g, h, _ = a.trace(1.0, budget=False)        # no sources: allocates and zeroes the rates
        torch.cuda.synchronize()
        g.copy_(torch.from_numpy(gamma.reshape(3, n, n, n)).cuda())
        torch.cuda.synchronize()
        dtn, dti = a.rt_timestep(0.1)
    f64 = lambda v: np.asarray(v, np.float64)
    odtn, odti = oracle.rt_timestep(p, f64(nH), f64(xHI), f64(xHeI), f64(xHeII), f64(T), f64(gamma[0]), 0.1)
    assert np.isfinite(odtn) and np.isfinite(odti)
    assert abs(dtn / odtn - 1) < 1e-5, (dtn, odtn)
    assert abs(dti / odti - 1) < 1e-5, (dti, odti)


def test_clump_test3_against_printed_results():
    """The paper's Test 3 (Sec. 3.4) at full size, 15 Myr, graph-stepped: the
    I-front along the line through the clump centre reaches x_HI = 0.5 near
    r/L = 0.8; the photo-heated gas outside the clump is above 3e4 K, the gas
    in the clump below 2e4 K; the shadow behind the clump stays neutral and
    the thin gas in front is ionised."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))["test3_clump"]
    w = W.clump_test3()
    with P.Arc(w.n, w.box_cm, w.params()) as a:
        a.set_fields(w.nH, w.xHI, w.xHeI, w.xHeII, w.T)
        a.add_sources(w.src_pos, w.src_ndot)
        for _ in range(w.nsteps):
            a.step(w.dt_s)
        x, _, _, T = a.get_fields()
    axis = lambda f: 0.25 * (f[:, 63, 63] + f[:, 63, 64] + f[:, 64, 63] + f[:, 64, 64])
    xa, Ta = axis(x), axis(T)
    rL = (np.arange(w.n) + 0.5) / w.n
    k = np.where((rL > 0.6) & (xa > 0.5))[0][0]
    assert abs(rL[k] - gold["ifront_x_half_r_over_L"]) < 0.05, rL[k]
    assert (Ta[(rL > 0.05) & (rL < 0.55)] > gold["T_outside_clump_above_K"]).all()
    assert (Ta[(rL > 0.65) & (rL < 0.88)] < gold["T_inside_clump_below_K"]).all()
    assert (xa[rL > 0.9] > 0.5).all()
    assert (xa[(rL > 0.05) & (rL < 0.55)] < 1e-3).all()


def _oracle_chem_chunk(args):
    """One slice of cells through the FP64 oracle's chemistry (a spawned worker;
    the inputs are memory-mapped FP32 arrays, so workers share one copy)."""
    d, params, dt, lo, hi = args
    import os
    import oracle as O
    ld = lambda name: np.load(os.path.join(d, name + ".npy"), mmap_mode="r")
    s = slice(lo, hi)
    f = lambda a: np.asarray(a, np.float64)
    x0, g, h = ld("x0"), ld("g"), ld("h")
    r = O.chem(params, f(ld("nH")[s]), f(x0[0, s]), f(x0[1, s]), f(x0[2, s]), f(ld("T0")[s]), f(g[:, s]),
               f(h[:, s]), dt)
    return lo, [np.asarray(a, np.float32) for a in r[:4]], int(r[5])


def test_full_size_cosmic_256_chemistry_every_cell(tmp_path):
    """The 256^3 benchmark field after three graph-replayed steps (fronts around
    1000 sources, helium ionising next to the bright ones): one chemistry update
    on the GPU against the oracle's on every one of the 16.7M cells, with the
    rates the GPU traced.  The oracle runs in worker processes started with
    spawn, one slice of cells each."""
    import multiprocessing as mp
    import os
    w = W.cosmic_256()
    with P.Arc(w.n, w.box_cm, w.params()) as a:
        a.set_fields(w.nH, w.xHI, w.xHeI, w.xHeII, w.T)
        a.add_sources(w.src_pos, w.src_ndot)
        for _ in range(3):
            a.step(w.dt_s)
        state = a.get_fields()
        g, h, _ = a.trace(w.dt_s, budget=True)          # budget=True waits for the rates
        g = g.cpu().numpy().reshape(3, -1)
        h = h.cpu().numpy().reshape(3, -1)
        a.set_fields(w.nH, *state)
        a.chem(w.dt_s)
        st = a.stats()
        out = a.get_fields()
    assert st["chem_capped"] == 0 and st["chem_fp64_substeps"] > 0
    f32 = lambda x: np.ascontiguousarray(np.asarray(x, np.float32).reshape(-1))
    d = str(tmp_path)
    for name, arr in (("nH", f32(w.nH)), ("x0", np.stack([f32(s) for s in state[:3]])), ("T0", f32(state[3])),
                      ("g", g.astype(np.float32)), ("h", h.astype(np.float32))):
        np.save(os.path.join(d, name + ".npy"), arr)
    n3 = w.n ** 3
    step = n3 // 64
    ox = [np.zeros(n3, np.float32) for _ in range(4)]
    capped = 0
    jobs = [(d, w.params(), w.dt_s, i, min(i + step, n3)) for i in range(0, n3, step)]
    with mp.get_context("spawn").Pool(max(1, min(16, len(os.sched_getaffinity(0))))) as pool:
        for lo, res, c in pool.imap_unordered(_oracle_chem_chunk, jobs):
            for k in range(4):
                ox[k][lo:lo + res[k].size] = res[k]
            capped += c
    f = lambda x: np.asarray(x, np.float64).reshape(-1)
    assert capped == 0
    for k in range(3):
        assert np.max(np.abs(f(out[k]) - ox[k])) < X_ATOL, k
    assert np.max(np.abs(f(out[3]) / ox[3] - 1)) < T_RTOL
