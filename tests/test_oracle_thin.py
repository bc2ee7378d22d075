"""Pins of the oracle's optically thin approximation (Sec. 2.6) and of its
anisotropic escape masks (Sec. 2.2), against closed forms and the plain trace.

* in a uniform medium every ray reaches optical depth 0.1 in the softest group
  at distance 0.1 / kappa, so the thin radius is exactly that;
* rays launched at R in a transparent box form the tree of an independent walk
  (a ray at or beyond its split distance splits at once), and the next radius
  is the smallest exit distance of its leaves;
* beyond R the thin trace differs from the plain one only by the photons the
  plain rays lost inside R: the ratio of the rates is exp(kappa R) per cell;
* inside R the fill reproduces the shell-averaged traced rates once their
  attenuation exp(-kappa r) is removed (Eq. ion in the small-tau limit);
* masks: complementary masks add up to the unmasked trace, the launched
  photons are the open fraction, and one open pixel lights its own cone.
"""
import math

import numpy as np
import pytest

import oracle
from test_oracle_trace import exit_distance, fields, uniform_params


def _trace(p, n, kappa_scale, o, ndot=1e48, **kw):
    nH, x, z, z2 = fields(n)
    return oracle.trace(p, nH, x * kappa_scale, z, z2, np.asarray(o, float)[None, :], np.array([[ndot]]), **kw)


@pytest.mark.parametrize("o,k", [((16.5, 16.5, 16.5), 0.01), ((10.25, 19.5, 14.75), 0.02)])
def test_thin_radius_uniform_closed_form(o, k):
    n = 32
    p = uniform_params(n, k)
    r = _trace(p, n, 1.0, o)
    assert abs(r["r_thin"][0] - 0.1 / k) < 1e-12 * (0.1 / k)


def test_thin_radius_uses_softest_group():
    """Two groups listed hardest first: the radius follows the lower-energy one."""
    n = 32
    p = uniform_params(n, 0.0, G=2)
    p["E_group_eV"] = [40.0, 20.0]
    p["sigma"][0] = [0.004 / 1e20, 0.02 / 1e20]     # kappa per cell 0.004 (hard), 0.02 (soft)
    nH, x, z, z2 = fields(n)
    r = oracle.trace(p, nH, x, z, z2, np.array([[16.5, 16.5, 16.5]]), np.array([[1e48, 1e48]]))
    assert abs(r["r_thin"][0] - 0.1 / 0.02) < 1e-12 * 5.0


def thin_tree(p, o, n, R):
    """Leaves and immediate splits of rays launched at R in a transparent box,
    built independently: a ray starting outside the box escapes there; one at
    or beyond its split distance splits at once; else it escapes at its exit
    distance if that comes before the split distance, or splits there."""
    recs = []

    def walk(l, pix, r0):
        u = oracle.pix2vec(l, pix)
        x = o + r0 * u
        if np.any(np.floor(x) < 0) or np.any(np.floor(x) >= n):
            recs.append((l, pix, oracle.END_ESCAPE, r0))
            return
        rs = oracle.r_split(p, l) if l < p["l_max"] else np.inf
        if r0 >= rs:
            recs.append((l, pix, oracle.END_SPLIT, r0))
            for k in range(4):
                walk(l + 1, 4 * pix + k, r0)
            return
        d = exit_distance(o, u, n)
        if d <= rs:
            recs.append((l, pix, oracle.END_ESCAPE, d))
        else:
            recs.append((l, pix, oracle.END_SPLIT, rs))
            for k in range(4):
                walk(l + 1, 4 * pix + k, rs)

    for q in range(48):
        walk(1, q, R)
    return recs


@pytest.mark.parametrize("o,R", [((16.5, 16.5, 16.5), 5.3), ((9.25, 20.5, 13.75), 3.1)])
def test_thin_start_tree_and_escape_radius(o, R):
    n = 32
    p = uniform_params(n, 1e-9)
    o = np.array(o)
    r = _trace(p, n, 1.0, o, r_start=[R], records=True)
    want = thin_tree(p, o, n, R)
    got = sorted((int(a["level"]), int(a["pix"]), int(a["end"]), float(a["r1"])) for a in r["recs"])
    want = sorted(want)
    assert len(got) == len(want)
    for g, w in zip(got, want):
        assert g[:3] == w[:3] and abs(g[3] - w[3]) < 1e-9, (g, w)
    # immediate splits trace no cell
    imm = [a for a in r["recs"] if a["end"] == oracle.END_SPLIT and a["r1"] == R]
    assert imm and all(int(a["visits"]) == 0 for a in imm)
    # no ray reaches tau = 0.1: the next radius is the smallest leaf exit distance
    leaves = [w[3] for w in want if w[2] == oracle.END_ESCAPE]
    assert abs(r["r_thin"][0] - min(leaves)) < 1e-9


@pytest.mark.parametrize("R", [4.0, 7.5])
def test_thin_trace_beyond_radius_is_the_plain_one_unattenuated(R):
    n = 32
    k = 0.01
    p = uniform_params(n, k)
    o = np.array([16.5, 15.25, 16.75])
    plain = _trace(p, n, 1.0, o)
    thin = _trace(p, n, 1.0, o, r_start=[R])
    c = np.indices((n, n, n)).reshape(3, -1).T
    near = np.clip(o, c, c + 1)                       # nearest point of each cell
    dmin = np.sqrt(((near - o) ** 2).sum(1))
    m = dmin > R + 1e-6
    g0 = plain["gamma"][0].ravel()[m]
    g1 = thin["gamma"][0].ravel()[m]
    assert (g0 > 0).all()
    assert np.abs(g1 / g0 - math.exp(k * R)).max() < 1e-10
    # rays launched at R carry every photon: the ray budget still closes
    em, ab, es = thin["budget"]
    assert abs(em - 1e48) < 1e-12 * 1e48 and abs(em - ab - es) < 1e-9 * em


def test_thin_fill_matches_traced_small_tau_limit():
    n = 32
    k = 0.01
    R = 8.0
    p = uniform_params(n, k)
    o = np.array([16.5, 16.5, 16.5])
    plain = _trace(p, n, 1.0, o)
    thin = _trace(p, n, 1.0, o, r_start=[R])
    c = np.indices((n, n, n)).reshape(3, -1).T + 0.5
    rc = np.sqrt(((c - o) ** 2).sum(1))
    g0 = plain["gamma"][0].ravel() * np.exp(k * rc)   # traced, attenuation removed
    g1 = thin["gamma"][0].ravel()
    for lo, hi in [(2.0, 4.0), (4.0, 6.0), (6.0, 7.5)]:
        sh = (rc > lo) & (rc < hi)
        ratio = g1[sh].sum() / g0[sh].sum()
        assert abs(ratio - 1.0) < 0.03, (lo, hi, ratio)
    # photons taken by the fill: S tau(R) for a uniform sphere, within the
    # cell discretisation of the sphere
    assert abs(thin["thin_photons"] / (1e48 * k * R) - 1.0) < 0.08


def test_thin_zero_radius_is_the_plain_trace():
    n = 24
    p = uniform_params(n, 0.3)
    o = (11.3, 12.6, 9.9)
    a = _trace(p, n, 1.0, o, records=True)
    b = _trace(p, n, 1.0, o, r_start=[0.0], records=True)
    assert np.array_equal(a["gamma"], b["gamma"]) and a["nrec"] == b["nrec"]
    assert b["thin_photons"] == 0.0


def _two_sources():
    n = 24
    p = uniform_params(n, 0.2)
    nH, x, z, z2 = fields(n)
    rng = np.random.Generator(np.random.PCG64(11))
    x = x * rng.uniform(0.2, 1.0, x.shape)
    pos = np.array([[6.3, 12.1, 17.4], [15.2, 8.8, 5.6]])
    ndot = np.array([[1e48], [3e48]])
    return p, (nH, x, z, z2), pos, ndot


def test_complementary_masks_add_up():
    p, f, pos, ndot = _two_sources()
    rng = np.random.Generator(np.random.PCG64(5))
    m = rng.integers(0, 2, (2, 48)).astype(bool)
    m[1, :40] = True                                   # different open counts per source
    full = oracle.trace(p, *f, pos, ndot)
    a = oracle.trace(p, *f, pos, ndot, open_mask=m, records=True)
    b = oracle.trace(p, *f, pos, ndot, open_mask=~m)
    g = full["gamma"]
    assert np.abs(a["gamma"] + b["gamma"] - g).max() < 1e-12 * g.max()
    frac = (m * ndot).sum() / 48.0
    assert abs(a["budget"][0] - frac) < 1e-9 * frac
    assert abs(a["budget"][0] + b["budget"][0] - ndot.sum()) < 1e-9 * ndot.sum()
    blocked = a["recs"][a["recs"]["end"] == oracle.END_BLOCKED]
    assert len(blocked) == (~m).sum()
    assert all(not m[int(q["src"]), int(q["pix"])] and q["visits"] == 0 and q["level"] == 1 for q in blocked)


@pytest.mark.parametrize("q", [5, 22, 40])
def test_single_open_pixel_lights_its_cone(q):
    """The photon-weighted mean direction of the deposits lies in the open pixel."""
    n = 32
    p = uniform_params(n, 0.05)
    o = np.array([16.3, 16.6, 16.45])
    m = np.zeros((1, 48), bool)
    m[0, q] = True
    r = _trace(p, n, 1.0, o, open_mask=m)
    g = r["gamma"][0].ravel()
    c = np.indices((n, n, n)).reshape(3, -1).T + 0.5
    v = ((c - o) / np.linalg.norm(c - o, axis=1)[:, None] * g[:, None]).sum(0)
    assert oracle.vec2pix(1, v) == q
    assert abs(r["budget"][0] - 1e48 / 48) < 1e-12 * 1e48


def test_thin_ledger_matches_the_cell_rates_with_helium():
    """Photons absorbed in the cells, rebuilt from the per-absorber rates
    (Gamma_s n_s V summed), equal the rays' absorbed photons plus the fill's
    ledger, with three absorbers and three groups."""
    import workloads as W
    w = W.thermal_128(n=24, box_kpc=6.6 * 24 / 128)
    w.src_pos = W.quantise_pos([[8.3, 12.7, 10.1], [15.5, 6.2, 17.75]])
    w.src_ndot = np.vstack([w.src_ndot[0], 0.5 * w.src_ndot[0]])
    xs = W.ionised_bubbles(w, 4.0)
    d = lambda a: np.asarray(a, np.float64)
    p = w.params()
    r = oracle.trace(p, d(w.nH), *[d(x) for x in xs], w.src_pos, w.src_ndot, r_start=[3.5, 2.25])
    em, ab, es = r["budget"]
    assert abs(em - ab - es) < 1e-9 * em and r["thin_photons"] > 0
    y = w.Y / (4 * (1 - w.Y))
    nH = d(w.nH)
    ns = np.stack([nH * d(xs[0]), y * nH * d(xs[1]), y * nH * d(xs[2])])
    cells = (r["gamma"] * ns).sum() * (w.box_cm / w.n) ** 3
    assert abs(cells - (ab + r["thin_photons"])) < 1e-9 * cells


def test_masks_and_thin_radii_are_refused_together():
    n = 16
    p = uniform_params(n, 0.1)
    with pytest.raises(ValueError):
        _trace(p, n, 1.0, (8.3, 8.6, 8.1), r_start=[2.0], open_mask=np.ones((1, 48), bool))
