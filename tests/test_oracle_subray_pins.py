"""Pins of the oracle's sub-ray system model (no GPU): each bin is R parallel lines spread
uniformly across its width, the ray-driven model with several parallel rays per detector pair of
the paper's simulations (Sec. IV-A, 32 rays there).

Checked against: rows of a dense matrix built by clipping every sub-line against every pixel
square; the exact count of sub-lines inside a pixel column for views along an axis; the strip
integral (the area of the bin's strip inside the pixel over the bin width) as R grows, computed
in closed form; adjointness; and R = 1 giving the one-line model.
"""
import math

import numpy as np
import pytest

import oracle
from test_oracle_pins import _dirs


def clip_length(n, c, s, r, x0, y0):
    """Length of the line {X c + Y s = r} inside the half-open square [x0, x0+1) x [y0, y0+1)."""
    lo, hi = -np.inf, np.inf
    if s == 0.0:
        if not (x0 <= r * c < x0 + 1):
            return 0.0
    else:
        t1, t2 = (r * c - x0) / s, (r * c - x0 - 1) / s
        lo, hi = max(lo, min(t1, t2)), min(hi, max(t1, t2))
    if c == 0.0:
        if not (y0 <= r * s < y0 + 1):
            return 0.0
    else:
        t1, t2 = (y0 - r * s) / c, (y0 + 1 - r * s) / c
        lo, hi = max(lo, min(t1, t2)), min(hi, max(t1, t2))
    return max(0.0, hi - lo)


@pytest.mark.parametrize("n,V,nb,rho,R", [(8, 8, 13, 1.0, 4), (8, 7, 12, 0.8, 5), (6, 9, 11, 1.3, 32)])
def test_subray_rows_match_dense_clipping(n, V, nb, rho, R):
    g = oracle.geom(n, 1, V, nb, 1, pixel_mm=1.0, bin_mm=rho, subrays=R)
    dirs = _dirs(V)
    for v in range(V):
        c, s = dirs[v]
        for b in range(nb):
            rb = (b - (nb - 1) / 2.0) * rho
            want = np.zeros(n * n)
            for k in range(R):
                r = rb + ((k + 0.5) / R - 0.5) * rho
                for iy in range(n):
                    for ix in range(n):
                        want[iy * n + ix] += clip_length(n, c, s, r, ix - n / 2.0, iy - n / 2.0) / R
            pix, ln = oracle.bin_pieces(g, v, b)
            got = np.zeros(n * n)
            np.add.at(got, pix, ln)
            np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_axis_view_counts_sub_lines_in_each_column():
    """View 0 (lines X = r): a pixel column holds (number of sub-lines with X in [x0, x0+1)) / R
    of unit length per pixel of the column."""
    n, nb, rho, R = 8, 15, 0.7, 32
    g = oracle.geom(n, 1, 4, nb, 1, pixel_mm=1.0, bin_mm=rho, subrays=R)
    for b in range(nb):
        rb = (b - (nb - 1) / 2.0) * rho
        xs = rb + ((np.arange(R) + 0.5) / R - 0.5) * rho
        pix, ln = oracle.bin_pieces(g, 0, b)
        got = np.zeros(n * n)
        np.add.at(got, pix, ln)
        for ix in range(n):
            x0 = ix - n / 2.0
            cnt = np.count_nonzero((xs >= x0) & (xs < x0 + 1))
            np.testing.assert_allclose(got.reshape(n, n)[:, ix], cnt / R, rtol=0, atol=1e-12)


def _chord_integral(c, s, x0, y0, a, b):
    """Integral over r in [a, b] of the length of {X c + Y s = r} inside [x0, x0+1] x [y0, y0+1]
    for an oblique direction (c, s != 0): the chord length is a trapezoid in r whose corners are
    the projections of the square's vertices; integrated piecewise (linear pieces, exactly)."""
    p = sorted([x0 * c + y0 * s, (x0 + 1) * c + y0 * s, x0 * c + (y0 + 1) * s,
                (x0 + 1) * c + (y0 + 1) * s])
    top = 1.0 / max(abs(c), abs(s))

    def chord(r):
        if r <= p[0] or r >= p[3]:
            return 0.0
        if r < p[1]:
            return top * (r - p[0]) / (p[1] - p[0])
        if r <= p[2]:
            return top
        return top * (p[3] - r) / (p[3] - p[2])

    pts = sorted(set([a, b] + [x for x in p if a < x < b]))
    return sum(0.5 * (chord(u) + chord(w)) * (w - u) for u, w in zip(pts[:-1], pts[1:]))


def test_many_sub_rays_approach_the_strip_integral():
    """As R grows the bin's row tends to (area of its strip inside the pixel) / bin width."""
    n, V, nb, rho = 6, 9, 11, 1.0
    R = 4096
    g = oracle.geom(n, 1, V, nb, 1, pixel_mm=1.0, bin_mm=rho, subrays=R)
    dirs = _dirs(V)
    for v in (1, 2, 4):
        c, s = dirs[v]
        for b in (2, 5, 8):
            rb = (b - (nb - 1) / 2.0) * rho
            pix, ln = oracle.bin_pieces(g, v, b)
            got = np.zeros(n * n)
            np.add.at(got, pix, ln)
            for iy in range(n):
                for ix in range(n):
                    want = _chord_integral(c, s, ix - n / 2.0, iy - n / 2.0, rb - rho / 2, rb + rho / 2) / rho
                    assert abs(got[iy * n + ix] - want) < 2e-6, (v, b, ix, iy, got[iy * n + ix], want)


def test_subray_adjointness_and_single_line_limit():
    n, P, V, nb, M = 20, 2, 18, 29, 3
    g = oracle.geom(n, P, V, nb, M, pixel_mm=1.5, bin_mm=1.5, sens=2.0, subrays=8)
    rng = np.random.default_rng(3)
    for i in range(M):
        x = rng.uniform(0, 1, (P, n, n))
        y = rng.uniform(0, 1, (P, oracle.subset_size(g, i), nb))
        lhs = np.vdot(oracle.forward(g, i, x), y)
        rhs = np.vdot(x, oracle.back(g, i, y))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    g1 = oracle.geom(n, P, V, nb, M, pixel_mm=1.5, bin_mm=1.5, sens=2.0, subrays=1)
    x = rng.uniform(0, 1, (P, n, n))
    np.testing.assert_array_equal(oracle.forward(g1, -1, x),
                                  oracle.forward(oracle.geom(n, P, V, nb, M, 1.5, 1.5, 2.0), -1, x))
    # the sub-ray model blurs: it differs from the one-line model
    assert np.abs(oracle.forward(g, -1, x) - oracle.forward(g1, -1, x)).max() > 1e-3
