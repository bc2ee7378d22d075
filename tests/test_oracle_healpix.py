"""Pins of the oracle's HEALPix nested pix2vec / vec2pix (Sec. 2.1; Gorski et al. 2005).

Checked against what the pixelisation fixes independently of the nested index
arithmetic: ring latitudes and ring sizes, equal spacing in longitude, equal
areas (Monte Carlo), the nested parent/child relation and symmetry.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")


def all_vecs(level):
    npix = 12 * 4 ** level
    return np.array([oracle.pix2vec(level, p) for p in range(npix)])


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_roundtrip(level):
    npix = 12 * 4 ** level
    for p in range(npix):
        assert oracle.vec2pix(level, oracle.pix2vec(level, p)) == p


@pytest.mark.parametrize("level", [1, 2, 3, 4])
def test_ring_latitudes_and_sizes(level):
    """Ring i (1 <= i <= 4 ns - 1) sits at z = 1 - i^2/(3 ns^2) in the north cap,
    z = 4/3 - 2 i/(3 ns) in the belt, mirrored in the south; caps hold 4 i pixels
    per ring and belt rings 4 ns."""
    ns = 2 ** level
    v = all_vecs(level)
    z = v[:, 2]
    assert np.allclose((v ** 2).sum(1), 1.0, atol=1e-14)
    expect = {}
    for i in range(1, 4 * ns):
        if i < ns:
            zi, cnt = 1 - i * i / (3 * ns * ns), 4 * i
        elif i <= 3 * ns:
            zi, cnt = 4 / 3 - 2 * i / (3 * ns), 4 * ns
        else:
            j = 4 * ns - i
            zi, cnt = -(1 - j * j / (3 * ns * ns)), 4 * j
        expect[i] = (zi, cnt)
    used = np.zeros(len(z), bool)
    for i, (zi, cnt) in expect.items():
        m = np.abs(z - zi) < 1e-12
        assert m.sum() == cnt, (i, m.sum(), cnt)
        assert not (used & m).any()
        used |= m
        # equally spaced in longitude; first pixel offset is half a step in the
        # caps and on odd-shifted belt rings
        phi = np.sort(np.mod(np.arctan2(v[m, 1], v[m, 0]), 2 * np.pi))
        step = 2 * np.pi / cnt
        assert np.allclose(np.diff(phi), step, atol=1e-12)
        off = phi[0] / step
        if i < ns or i > 3 * ns:
            assert abs(off - 0.5) < 1e-9
        elif (i - ns) % 2 == 0:
            assert abs(off - 0.5) < 1e-9
        else:
            assert min(abs(off), abs(off - 1.0)) < 1e-9
    assert used.all()


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_symmetry_sum_zero(level):
    assert np.abs(all_vecs(level).sum(0)).max() < 1e-11


def test_equal_area_monte_carlo():
    """Uniform random directions land in the 192 level-2 pixels with equal
    probability (chi^2 test)."""
    rng = np.random.Generator(np.random.PCG64(11))
    m = 200_000
    v = rng.standard_normal((m, 3))
    counts = np.zeros(192)
    for x in v:
        counts[oracle.vec2pix(2, x)] += 1
    e = m / 192
    chi2 = ((counts - e) ** 2 / e).sum()
    # 191 dof: mean 191, sd ~ 19.5; 5 sigma bound
    assert chi2 < 191 + 5 * 19.6, chi2


@pytest.mark.parametrize("level", [1, 2, 3])
def test_children_nest_inside_parent(level):
    """Children 4p..4p+3 of pixel p lie in p: vec2pix at the parent level of a
    child centre returns p, and each child centre is nearer p's centre than any
    other parent centre."""
    parents = all_vecs(level)
    for p in range(12 * 4 ** level):
        for k in range(4):
            c = oracle.pix2vec(level + 1, 4 * p + k)
            assert oracle.vec2pix(level, c) == p
            d = parents @ c
            assert int(np.argmax(d)) == p
