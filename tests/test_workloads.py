"""Host checks of the seeded input generators (no method arithmetic lives
here): source positions as drawn or on the FP32 grid, the ionised-sphere state against a brute-force
distance test, and reproducibility from the seed."""
import numpy as np
import pytest

import workloads as W


def test_positions_as_drawn_or_on_the_fp32_grid():
    """By default source positions are the FP64 draws (the tracer carries them as
    FP32 pairs); quantise=True rounds them to 2^-12 cell, exact in FP32."""
    w = W.cosmic(n=32, nsrc=20, seed=3)
    q = W.cosmic(n=32, nsrc=20, seed=3, quantise=True)
    assert ((w.src_pos >= 0) & (w.src_pos < w.n)).all()
    assert not np.array_equal(w.src_pos.astype(np.float32).astype(np.float64), w.src_pos)
    assert np.array_equal(q.src_pos.astype(np.float32).astype(np.float64), q.src_pos)
    assert np.abs(q.src_pos - w.src_pos).max() <= 2.0 ** -13


def test_cosmic_field_is_seeded():
    a = W.cosmic(n=32, nsrc=10, seed=7)
    b = W.cosmic(n=32, nsrc=10, seed=7)
    c = W.cosmic(n=32, nsrc=10, seed=8)
    assert np.array_equal(a.nH, b.nH) and np.array_equal(a.src_pos, b.src_pos)
    assert not np.array_equal(a.nH, c.nH)
    assert abs(a.nH.mean() / 2e-4 - 1.0) < 1e-6


@pytest.mark.parametrize("radius", [0.7, 3.0, 9.5, 100.0])
def test_ionised_bubbles_against_brute_force(radius):
    w = W.cosmic(n=24, nsrc=6, seed=2)
    xHI, xHeI, xHeII = W.ionised_bubbles(w, radius)
    n = w.n
    c = np.indices((n, n, n)).reshape(3, -1).T + 0.5
    inside = np.zeros(n ** 3, bool)
    for o in w.src_pos:
        inside |= ((c - o) ** 2).sum(1) < radius * radius
    inside = inside.reshape(n, n, n)
    assert np.array_equal(xHI < 1e-3, inside)
    assert (xHI[inside] == np.float32(1e-4)).all() and (xHeII[inside] == np.float32(0.05)).all()
    assert np.array_equal(xHI[~inside], w.xHI[~inside])
