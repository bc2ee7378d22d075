"""Sec. 3.6 methodology test of the geometric correction (Sec. 2.5, Eqs.
correction and correction2), on the oracle.

A Stromgren sphere (pure H, isothermal, case B, R_S ~ 16 cells) grown by trace
+ chemistry for ~3 recombination times with four treatments of a ray's cone
near cell faces: none; f_c with the secondary f'_c to the nearest neighbour
(photon conserving); f_c alone; f_c squared alone (the form of the method the
paper modifies).  The paper finds that f_c and f_c^2 shrink the ionised region
by roughly 5 and 10 per cent and that adding f'_c restores its size.  Here, at
Phi = 3 rays per cell face, f_c must shrink the volume-equivalent front radius
by 2-8 per cent, f_c^2 by 5-15 per cent and by more than f_c, and f_c + f'_c
must stay within 1.5 per cent of the uncorrected run; at Phi = 1 (pixels wider
than cells, so more segments are corrected) each shrink is larger than at
Phi = 3 and f_c + f'_c still restores the radius within 2 per cent.  The
photon-conserving variant credits every absorbed photon to some cell; the two
primary-only variants credit fewer.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

NDOT = 4e48      # R_S = 15.7 cells at the Stromgren workload's density and cell size
NSTEPS = 40      # 40 Myr = 3.3 t_rec


def front_radius(w, phi, mode):
    p = w.params()
    p["phi"] = phi
    p["geo_corr"] = mode
    xHI, *_ = oracle.run(p, w, NSTEPS)
    return (3 * (1 - xHI).sum() / (4 * math.pi)) ** (1 / 3)


@pytest.fixture(scope="module")
def radii():
    w = W.stromgren_32(n=48)
    w.src_ndot = np.array([[NDOT]])
    return {phi: {m: front_radius(w, phi, m) for m in (0, 1, 2, 3)} for phi in (1.0, 3.0)}


def test_correction_variants_shrink_or_restore_the_front(radii):
    shrink = {phi: {m: 1 - r[m] / r[0] for m in (1, 2, 3)} for phi, r in radii.items()}
    s3 = shrink[3.0]
    assert 0.02 < s3[2] < 0.08, s3
    assert 0.05 < s3[3] < 0.15 and s3[3] > s3[2], s3
    assert abs(s3[1]) < 0.015, s3
    s1 = shrink[1.0]
    assert s1[2] > s3[2] and s1[3] > s3[3], (s1, s3)
    assert abs(s1[1]) < 0.02, s1


def test_only_the_secondary_variant_conserves_photons():
    """Rates rebuilt into photons per cell (Gamma n_HI V) against the photons
    the rays lost: equal with f_c + f'_c, short with the primary factor alone."""
    w = W.stromgren_32(n=24)
    w.src_ndot = np.array([[NDOT]])
    xHI = np.full(w.nH.shape, 0.3)
    V = (w.box_cm / w.n) ** 3
    credited = {}
    for mode in (1, 2, 3):
        p = w.params()
        p["phi"] = 1.0
        p["geo_corr"] = mode
        tr = oracle.trace(p, w.nH.astype(np.float64), xHI, w.xHeI.astype(np.float64),
                          w.xHeII.astype(np.float64), w.src_pos, w.src_ndot)
        em, ab, es = tr["budget"]
        cells = float((tr["gamma"][0] * w.nH * xHI * V).sum())
        credited[mode] = cells / ab
    assert abs(credited[1] - 1) < 1e-9, credited
    assert credited[3] < credited[2] < 0.99, credited
