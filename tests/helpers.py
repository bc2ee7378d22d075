"""Shared test helpers: run the CUDA path and the oracle on the same inputs and
compare them.  Tolerances (stated in the tests that use them):

* integer ray tree: split levels, end reasons and per-ray cell-visit counts
  equal, except for rays whose oracle decision margin lies inside the FP32
  band (64 ulps of the compared distance, 1e-4 relative for the photon
  threshold) and their descendants, which are counted and reported;
* Gamma and heating per absorber: relative 1e-4 wherever the oracle's value
  exceeds 1e-6 of its maximum;
* photon budget: |launched - absorbed - escaped| <= 1e-9 launched.
"""
from __future__ import annotations

import numpy as np

import oracle
import workloads as W

GEO_ULPS = 64
TERM_BAND = 1e-4
GAMMA_RTOL = 1e-4
GAMMA_FLOOR = 1e-6


def gpu_trace(w, xHI=None, xHeI=None, xHeII=None, records=False, rec_cap=1 << 22, dt=1.0,
              tuning=None, params=None, open_mask=None, thin_radii=None):
    """thin_radii: run with the optically thin approximation from these radii
    (Sec. 2.6); open_mask: emission mask [nsrc, 12*4^l_base] (Sec. 2.2)."""
    import torch
    import paper_1807_07094_gb300 as P
    p = dict(params or w.params())
    if thin_radii is not None:
        p["thin_approx"] = 1
    f32 = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))
    xHI = w.xHI if xHI is None else xHI
    xHeI = w.xHeI if xHeI is None else xHeI
    xHeII = w.xHeII if xHeII is None else xHeII
    with P.Arc(w.n, w.box_cm, p) as a:
        if tuning:
            a.set_tuning(*tuning)
        a.set_fields(f32(w.nH), f32(xHI), f32(xHeI), f32(xHeII), f32(w.T))
        a.add_sources(w.src_pos, w.src_ndot)
        if open_mask is not None:
            a.set_emission_mask(open_mask)
        if thin_radii is not None:
            a.set_thin_radii(thin_radii)
        buf = None
        if records:
            buf = torch.empty(rec_cap * P.REC_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
            a.set_records(buf.data_ptr(), rec_cap)
        g, h, b = a.trace(dt, budget=True)
        g = g.cpu().numpy().astype(np.float64)
        h = h.cpu().numpy().astype(np.float64)
        st = a.stats()
        r_thin = thin = None
        if thin_radii is not None:
            r_thin, thin = a.thin_radii(len(w.src_pos))
        recs = None
        if records:
            nrec = a.record_count()
            assert nrec <= rec_cap
            recs = buf[: nrec * P.REC_DTYPE.itemsize].cpu().numpy().view(P.REC_DTYPE)
    return dict(gamma=g, heat=h, budget=b, stats=st, recs=recs, r_thin=r_thin, thin_photons=thin)


def oracle_trace(w, xHI=None, xHeI=None, xHeII=None, records=False, params=None, open_mask=None,
                 r_start=None):
    p = params or w.params()
    xHI = w.xHI if xHI is None else xHI
    xHeI = w.xHeI if xHeI is None else xHeI
    xHeII = w.xHeII if xHeII is None else xHeII
    # the oracle sees exactly the FP32 values the GPU gets
    d = lambda a: np.asarray(np.asarray(a, np.float32), np.float64)
    return oracle.trace(p, d(w.nH), d(xHI), d(xHeI), d(xHeII), w.src_pos, w.src_ndot,
                        records=records, open_mask=open_mask, r_start=r_start)


def geo_band(r, n):
    return GEO_ULPS * 2.0 ** -23 * np.maximum(np.maximum(r, n), 1.0)


def compare_records(gpu_recs, orc_recs, n):
    """Compare ray trees key by key (source, level, pixel).

    A ray whose own visit count rests on an undecided tie (oracle geometric
    margin inside the band) may differ by that count only; a ray whose fate
    rests on one (photon threshold, or a box exit at the split distance) may
    also have a different subtree, so its descendants are not compared.
    Returns counts and the mismatching keys."""
    orc = {}
    fate = set()
    own = set()
    for a in orc_recs:
        key = (int(a["src"]), int(a["level"]), int(a["pix"]))
        orc[key] = a
        band = geo_band(a["r1"], n)
        if a["term_margin"] < TERM_BAND or a["exit_margin"] < band:
            fate.add(key)
        elif a["geo_margin"] < band:
            own.add(key)

    def ancestor_fate(key):
        s, l, p = key
        l -= 1
        p >>= 2
        while l >= 1:
            if (s, l, p) in fate:
                return True
            l -= 1
            p >>= 2
        return False

    gpu = {}
    dup = 0
    for a in gpu_recs:
        key = (int(a["src"]), int(a["level"]), int(a["pix"]))
        if key in gpu:
            dup += 1
        gpu[key] = a
    mism = []
    checked = skipped = 0
    for key, a in orc.items():
        if ancestor_fate(key):
            skipped += 1
            continue
        b = gpu.get(key)
        if key in fate or key in own:
            # undecided: the ray must exist; its count/end may differ
            if b is None and key in own:
                mism.append((key, None, "missing"))
            skipped += 1
            continue
        if b is None or int(b["visits"]) != int(a["visits"]) or int(b["end"]) != int(a["end"]):
            mism.append((key, None if b is None else (int(b["visits"]), int(b["end"])),
                         (int(a["visits"]), int(a["end"]), float(a["geo_margin"]),
                          float(a["term_margin"]), float(a["exit_margin"]))))
        checked += 1
    extra = [k for k in gpu if k not in orc and not ancestor_fate(k)]
    return dict(checked=checked, undecided=len(fate) + len(own), skipped=skipped,
                mismatches=mism, extra=extra, dup=dup, n_gpu=len(gpu_recs), n_orc=len(orc_recs))


def rate_errors(g_gpu, g_orc, floor=GAMMA_FLOOR, absorbers=None, min_photons=None):
    """Max relative error of the GPU rates over cells where the oracle exceeds
    floor * max (per species).  With absorbers (n_s V per species and cell)
    and min_photons, only cells where species s absorbs more than min_photons
    per second are compared (rate fields only; for heating the same cells)."""
    out = []
    for s in range(g_orc.shape[0]):
        o = g_orc[s]
        mx = o.max()
        if mx <= 0:
            out.append((0.0, 0, float(np.abs(g_gpu[s]).max())))
            continue
        m = o > floor * mx
        if absorbers is not None:
            m &= absorbers[s] * o > min_photons
        if not m.any():
            out.append((0.0, 0, {}))
            continue
        rel = np.abs(g_gpu[s][m] - o[m]) / o[m]
        i = int(np.argmax(rel))
        worst = dict(rel=float(rel[i]), orc_over_max=float(o[m][i] / mx), gpu=float(g_gpu[s][m][i]),
                     orc=float(o[m][i]), cell=np.argwhere(m)[i].tolist(),
                     n_over_1e4=int((rel > 1e-4).sum()), n_over_1e3=int((rel > 1e-3).sum()))
        out.append((float(rel.max()), int(m.sum()), worst))
    return out


def partly_ionised(w, seed, lo=-6.0, hi=0.0):
    """Random ionisation state on the workload's gas (log-uniform x_HI)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sh = w.nH.shape
    xHI = (10 ** rng.uniform(lo, hi, sh)).astype(np.float32)
    xHeI = (10 ** rng.uniform(lo, hi, sh)).astype(np.float32)
    xHeII = ((1 - xHeI) * rng.uniform(0, 1, sh)).astype(np.float32)
    if w.Y == 0:
        xHeI[:] = 0
        xHeII[:] = 0
    return xHI, xHeI, xHeII
