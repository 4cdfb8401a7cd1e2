"""Pins of the oracle's ring sampling (no GPU): the bins of one view as the lines of a detector
ring of radius Rd equally spaced in angle (the paper's scanner is a ring of 576 detectors,
Sec. IV-A), r_b = Rd sin(beta_b), with R sub-rays spread over each bin's width.

Checked against: rows of the dense clipping matrix at those offsets, written out here; the
symmetry and cos(beta) narrowing of the bins; a huge ring reducing to uniform bins; the sub-rays
summing to the strip of the bin's width; and adjointness.
"""
import math

import numpy as np
import pytest

import oracle
from test_oracle_pins import _dirs
from test_oracle_subray_pins import clip_length


def ring_offsets(nb, bin_mm, ring_mm):
    beta = (np.arange(nb) - (nb - 1) / 2.0) * bin_mm / ring_mm
    return ring_mm * np.sin(beta), bin_mm / ring_mm


@pytest.mark.parametrize("n,V,nb,bin_mm,ring_mm,R", [(8, 6, 15, 1.0, 6.0, 1), (8, 7, 13, 1.2, 5.0, 3),
                                                     (6, 5, 11, 0.9, 4.0, 8)])
def test_ring_rows_match_dense_clipping(n, V, nb, bin_mm, ring_mm, R):
    g = oracle.geom(n, 1, V, nb, 1, pixel_mm=1.0, bin_mm=bin_mm, subrays=R, ring_mm=ring_mm)
    r, db = ring_offsets(nb, bin_mm, ring_mm)
    dirs = _dirs(V)
    for v in range(V):
        c, s = dirs[v]
        for b in range(nb):
            beta = (b - (nb - 1) / 2.0) * db
            lo, hi = ring_mm * math.sin(beta - db / 2), ring_mm * math.sin(beta + db / 2)
            lines = [r[b]] if R == 1 else [lo + (k + 0.5) / R * (hi - lo) for k in range(R)]
            want = np.zeros(n * n)
            for rr in lines:
                for iy in range(n):
                    for ix in range(n):
                        want[iy * n + ix] += clip_length(n, c, s, rr, ix - n / 2.0, iy - n / 2.0) / len(lines)
            pix, ln = oracle.bin_pieces(g, v, b)
            got = np.zeros(n * n)
            np.add.at(got, pix, ln)
            np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_ring_bins_symmetric_and_narrowing():
    """Offsets are odd in b and their spacing is Rd (sin(beta + db) - sin(beta)), shrinking with
    |beta|; on view 0 (lines X = r) a pixel column's sensitivity follows the bins' density."""
    nb, bin_mm, ring_mm = 41, 1.0, 12.0
    r, db = ring_offsets(nb, bin_mm, ring_mm)
    np.testing.assert_allclose(r, -r[::-1], atol=1e-13)
    sp = np.diff(r)
    assert np.all(np.diff(sp[nb // 2:]) < 0) and np.all(np.diff(sp[:nb // 2]) > 0)
    n = 8
    g = oracle.geom(n, 1, 4, nb, 1, pixel_mm=1.0, bin_mm=bin_mm, ring_mm=ring_mm)
    for b in range(nb):
        pix, ln = oracle.bin_pieces(g, 0, b)
        if len(pix):
            # the line X = r_b lies in column floor(r_b + n/2) (half-open pixels)
            assert np.all(pix % n == int(math.floor(r[b] + n / 2.0)))


def test_huge_ring_is_uniform_bins():
    """(bin offsets off the pixel edges, where the half-open rule would flip a line's pixels for
    a 1e-9 change of its offset)"""
    n, P, V, nb, M = 12, 2, 9, 19, 3
    x = np.random.default_rng(0).uniform(0, 1, (P, n, n))
    for R in (1, 4):
        gu = oracle.geom(n, P, V, nb, M, pixel_mm=1.5, bin_mm=1.3, subrays=R)
        gr = oracle.geom(n, P, V, nb, M, pixel_mm=1.5, bin_mm=1.3, subrays=R, ring_mm=1e8)
        yu, yr = oracle.forward(gu, -1, x), oracle.forward(gr, -1, x)
        assert np.abs(yu - yr).max() <= 1e-9 * yu.max()


def test_ring_subrays_tend_to_the_strip_and_adjointness():
    n, V, nb, bin_mm, ring_mm = 8, 6, 17, 1.0, 7.0
    g = oracle.geom(n, 2, V, nb, 3, pixel_mm=1.0, bin_mm=bin_mm, subrays=2048, ring_mm=ring_mm)
    dirs = _dirs(V)
    _, db = ring_offsets(nb, bin_mm, ring_mm)
    from test_oracle_subray_pins import _chord_integral
    for v in (1, 2, 4):
        c, s = dirs[v]
        for b in (3, 8, 12):
            beta = (b - (nb - 1) / 2.0) * db
            lo, hi = ring_mm * math.sin(beta - db / 2), ring_mm * math.sin(beta + db / 2)
            pix, ln = oracle.bin_pieces(g, v, b)
            got = np.zeros(n * n)
            np.add.at(got, pix, ln)
            for iy in range(n):
                for ix in range(n):
                    want = _chord_integral(c, s, ix - n / 2.0, iy - n / 2.0, lo, hi) / (hi - lo)
                    assert abs(got[iy * n + ix] - want) < 3e-6
    g = oracle.geom(n, 2, V, nb, 3, pixel_mm=1.0, bin_mm=bin_mm, subrays=4, ring_mm=ring_mm)
    rng = np.random.default_rng(1)
    for i in range(3):
        x = rng.uniform(0, 1, (2, n, n))
        y = rng.uniform(0, 1, (2, oracle.subset_size(g, i), nb))
        lhs, rhs = np.vdot(oracle.forward(g, i, x), y), np.vdot(x, oracle.back(g, i, y))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
