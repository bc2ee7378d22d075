"""GPU parity of the emission masks (Sec. 2.2) and of the optically thin
approximation (Sec. 2.6) against the oracle, through the C ABI.

Tolerances (on top of those of the plain trace, see helpers.py):
* ray trees: as for the plain trace; blocked rays match exactly (end code 4,
  no visit); rays launched at the thin radius start from the same FP32 radius
  on both sides, and a start cell or an immediate split decided inside the
  FP32 band is undecided;
* thin radius: relative 1e-4 -- the crossing point is r + ln(N / N_0.1) /
  kappa_0 with the photon ratio in FP32, ~1e-7 / kappa_0 cells;
* rates: relative 1e-4 outside cells whose centre lies within 1e-4 R of a
  source's sphere (inside or outside is an FP32 decision there);
* thin-fill photons: relative 1e-3 (those boundary cells may fall either way).
"""
import numpy as np
import pytest

import workloads as W
from helpers import GAMMA_RTOL, compare_records, gpu_trace, oracle_trace, partly_ionised, rate_errors

pytestmark = pytest.mark.gpu

R_RTOL = 1e-4
FILL_RTOL = 1e-3


def bubbles(w, radius):
    return W.ionised_bubbles(w, radius)


def boundary_cells(w, radii):
    n = w.n
    c = np.indices((n, n, n)).reshape(3, -1).T + 0.5
    m = np.zeros(n ** 3, bool)
    for o, R in zip(w.src_pos, radii):
        if R > 0:
            r = np.sqrt(((c - o) ** 2).sum(1))
            m |= np.abs(r - R) < 1e-4 * R + 1e-4
    return m.reshape(n, n, n)


def check_rates(g, o, skip=None):
    for name in ("gamma", "heat"):
        a, b = g[name].copy(), o[name].copy()
        if skip is not None:
            a[:, skip] = 0.0
            b[:, skip] = 0.0
        errs = rate_errors(a, b)
        if name == "gamma":
            assert errs[0][1] > 0
        for s, (rel, cnt, worst) in enumerate(errs):
            assert rel <= GAMMA_RTOL, (name, s, cnt, worst)


def check_trees(g, o, n):
    c = compare_records(g["recs"], o["recs"], n)
    assert c["dup"] == 0
    assert not c["mismatches"], (len(c["mismatches"]), c["checked"], c["mismatches"][:5])
    assert not c["extra"], c["extra"][:5]
    assert c["undecided"] <= 0.05 * max(c["n_orc"], 1), c
    return c


def test_emission_mask_parity():
    w = W.cosmic(n=48, nsrc=8, sigma_ln=1.5, seed=5)
    xs = partly_ionised(w, seed=4, lo=-3, hi=0)
    rng = np.random.Generator(np.random.PCG64(21))
    m = rng.uniform(size=(len(w.src_pos), 48)) < rng.uniform(0.1, 0.9, (len(w.src_pos), 1))
    m[0, :] = True
    m[1, :] = False                       # a source with every direction blocked
    g = gpu_trace(w, *xs, records=True, open_mask=m)
    o = oracle_trace(w, *xs, records=True, open_mask=m)
    launched, absorbed, escaped, emitted = g["budget"]
    assert abs(launched - absorbed - escaped) <= 1e-9 * launched
    want = (m.sum(1) / 48.0 * w.src_ndot.sum(1)).sum()
    assert abs(launched - want) <= 1e-6 * want and abs(o["budget"][0] - want) <= 1e-9 * want
    assert abs(emitted - w.src_ndot.sum()) <= 1e-9 * emitted
    blocked = g["recs"][g["recs"]["end"] == 4]
    assert len(blocked) == (~m).sum() and (blocked["visits"] == 0).all()
    check_trees(g, o, w.n)
    check_rates(g, o)


def _thin_pair(w, xs, R_in):
    R_in = np.asarray(R_in, np.float32).astype(np.float64)   # both sides get the FP32 radii
    g = gpu_trace(w, *xs, records=True, thin_radii=R_in)
    o = oracle_trace(w, *xs, records=True, r_start=R_in)
    launched, absorbed, escaped, emitted = g["budget"]
    assert abs(launched - absorbed - escaped) <= 1e-9 * launched
    check_trees(g, o, w.n)
    check_rates(g, o, skip=boundary_cells(w, R_in))
    rel = np.abs(g["r_thin"] - o["r_thin"]) / np.maximum(o["r_thin"], 1e-30)
    assert (rel <= R_RTOL).all(), (g["r_thin"], o["r_thin"])
    if o["thin_photons"] > 0:
        assert abs(g["thin_photons"] - o["thin_photons"]) <= FILL_RTOL * o["thin_photons"]
    else:
        assert g["thin_photons"] == 0.0
    return g, o


def test_thin_radius_measured_from_the_source():
    """Radii 0: the plain trace, and the radius it measures."""
    w = W.stromgren_32()
    xs = bubbles(w, 7.0)
    g, o = _thin_pair(w, xs, [0.0])
    # rays leave the ionised cells (centres within 7) at 6-7 cells: the
    # radius sits just past that exit, where 0.1 is reached in neutral gas
    assert 6.0 < o["r_thin"][0] < 7.5
    assert g["stats"]["rays"] == len(o["recs"])


def test_thin_trace_from_measured_radius_pure_h():
    w = W.stromgren_32()
    xs = bubbles(w, 7.0)
    R1 = oracle_trace(w, *xs)["r_thin"]
    g, o = _thin_pair(w, xs, R1)
    assert o["thin_photons"] > 0
    # rays launched past the first split distances: immediate splits exist
    assert ((o["recs"]["visits"] == 0) & (o["recs"]["end"] == 1)).any()


def test_thin_trace_helium_many_sources():
    w = W.thermal_128(n=48, box_kpc=6.6 * 48 / 128)
    w.src_pos = W.quantise_pos([[12.3, 20.7, 30.1], [33.5, 14.2, 21.75], [24.1, 35.3, 9.6]])
    w.src_ndot = np.vstack([w.src_ndot[0], 0.4 * w.src_ndot[0], 2.0 * w.src_ndot[0]])
    xs = bubbles(w, 5.0)
    R1 = oracle_trace(w, *xs)["r_thin"]
    assert (R1 > 1.0).all()
    _thin_pair(w, xs, R1)
    # and radii that are not the measured ones (one source without a region)
    _thin_pair(w, xs, [3.3, 0.0, 6.1])


def test_masks_and_thin_mode_do_not_combine():
    import paper_1807_07094_gb300 as P
    w = W.stromgren_32()
    p = dict(w.params(), thin_approx=1)
    f32 = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))
    with P.Arc(w.n, w.box_cm, p) as a:
        a.set_fields(f32(w.nH), f32(w.xHI), f32(w.xHeI), f32(w.xHeII), f32(w.T))
        a.add_sources(w.src_pos, w.src_ndot)
        with pytest.raises(P.ArcError):
            a.set_emission_mask(np.ones((1, 48), bool))
        with pytest.raises(P.ArcError):
            a.set_thin_radii([1.0, 2.0])          # one radius per source
        a.set_thin_radii([2.5])
        a.trace(1.0)
        r, thin = a.thin_radii(1)
        assert r[0] > 0 and thin > 0
