"""Pins of the oracle's time-of-flight system model (no GPU): bin (v, b) split into T TOF bins
along the line, A_{(v,b,t) j} = A_{(v,b) j} h_t(tau_j), h_t the Gaussian timing kernel integrated
over TOF bin t at the position tau_j of pixel j's centre along the line (TOF data as in the
clinical reconstructions of Sec. IV-C).

Checked against: h_t written out here with math.erf (closed forms: the value at a bin centre,
mirror symmetry, the sharp-kernel limit); rows of the dense clipping matrix times those weights;
the TOF bins adding up to the plain model when they cover the image; adjointness; EM count
preservation; and L-BFGS-B on Phi built from the dense TOF matrix (Theorem 2).
"""
import math

import numpy as np
import pytest

import oracle
from test_oracle_pins import P, _dirs, dense_A


def h_ref(T, dtau, fwhm, t, tau):
    sigma = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    c = (t - 0.5 * (T - 1)) * dtau
    phi = lambda z: 0.5 * (1.0 + math.erf(z / math.sqrt(2.0)))
    return phi((tau - c + 0.5 * dtau) / sigma) - phi((tau - c - 0.5 * dtau) / sigma)


def test_tof_weight_closed_forms():
    g = oracle.geom(8, 1, 4, 11, 1, pixel_mm=2.0, tof_bins=7, tof_bin_mm=10.0, tof_fwhm_mm=25.0)
    sigma = 25.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    for t in range(7):
        c = (t - 3) * 10.0
        # at the bin centre: erf(dtau / (2 sqrt 2 sigma))
        assert abs(oracle.tof_weight(g, t, c) - math.erf(5.0 / (math.sqrt(2.0) * sigma))) < 1e-15
        for tau in (-61.3, -7.0, 0.0, 3.3, 44.1, 140.0):
            assert abs(oracle.tof_weight(g, t, tau) - h_ref(7, 10.0, 25.0, t, tau)) < 1e-14
            assert abs(oracle.tof_weight(g, t, tau) - oracle.tof_weight(g, 6 - t, -tau)) < 1e-15
    # the bins partition the line: the weights of all bins add up to the covered mass
    for tau in (-20.0, 0.0, 13.7):
        tot = sum(oracle.tof_weight(g, t, tau) for t in range(7))
        want = h_ref(1, 70.0, 25.0, 0, tau)
        assert abs(tot - want) < 1e-14
    # a sharp kernel is the indicator of the bin
    gs = oracle.geom(8, 1, 4, 11, 1, pixel_mm=2.0, tof_bins=7, tof_bin_mm=10.0, tof_fwhm_mm=1e-6)
    assert oracle.tof_weight(gs, 4, 12.0) == 1.0 and oracle.tof_weight(gs, 4, 16.0) == 0.0


@pytest.mark.parametrize("n,V,nb,T,dtau,fwhm", [(8, 6, 11, 5, 6.0, 9.0), (10, 7, 13, 9, 4.0, 15.0)])
def test_tof_rows_match_dense_clipping(n, V, nb, T, dtau, fwhm):
    """A_tof x from the oracle equals the dense clipping matrix weighted by h_t at pixel centres."""
    px = 1.5
    g = oracle.geom(n, 1, V, nb, 1, pixel_mm=px, sens=1.0, tof_bins=T, tof_bin_mm=dtau,
                    tof_fwhm_mm=fwhm)
    A = dense_A(n, V, nb) * px                                   # lengths in mm
    x = np.random.default_rng(n).uniform(0, 1, n * n)
    got = oracle.forward(g, -1, x.reshape(1, n, n))[0]          # [V][nb][T]
    dirs = _dirs(V)
    X = (np.arange(n) + 0.5 - n / 2.0)[None, :].repeat(n, 0).ravel()
    Y = (np.arange(n) + 0.5 - n / 2.0)[:, None].repeat(n, 1).ravel()
    for v in range(V):
        c, s = dirs[v]
        tau = (-X * s + Y * c) * px
        for t in range(T):
            w = np.array([h_ref(T, dtau, fwhm, t, tj) for tj in tau])
            want = A[v * nb:(v + 1) * nb] @ (w * x)
            np.testing.assert_allclose(got[v, :, t], want, rtol=1e-12, atol=1e-13)


def test_tof_bins_add_up_to_the_plain_model_and_adjointness():
    n, Pn, V, nb, M = 16, 2, 12, 23, 3
    kw = dict(pixel_mm=4.0, sens=1.3)
    g = oracle.geom(n, Pn, V, nb, M, tof_bins=25, tof_bin_mm=12.0, tof_fwhm_mm=30.0, **kw)
    g0 = oracle.geom(n, Pn, V, nb, M, **kw)
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (Pn, n, n))
    y = oracle.forward(g, -1, x)
    y0 = oracle.forward(g0, -1, x)
    assert np.abs(y.sum(-1) - y0).max() <= 1e-12 * y0.max()
    np.testing.assert_allclose(oracle.sensitivity(g), oracle.sensitivity(g0), rtol=1e-12)
    for i in range(M):
        yi = oracle.forward(g, i, x)
        r = rng.uniform(0, 1, yi.shape)
        lhs, rhs = np.vdot(yi, r), np.vdot(x, oracle.back(g, i, r))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # the TOF bins resolve position along the line: they differ from the plain model's split
    assert np.abs(y[..., 12] - y0 / 25).max() > 0.1 * y0.max() / 25


def test_tof_em_count_preservation():
    n, V, nb = 12, 10, 17
    g = oracle.geom(n, 1, V, nb, 1, pixel_mm=3.0, sens=2.0, tof_bins=9, tof_bin_mm=8.0,
                    tof_fwhm_mm=20.0)
    rng = np.random.default_rng(3)
    ones = oracle.forward(g, -1, np.ones((1, n, n)))
    counts = np.where(ones > 1e-6, rng.integers(1, 40, ones.shape), 0).astype(np.int32)
    gamma = np.full(ones.shape, 1e-30, np.float32)
    sens_img = oracle.back(g, -1, np.ones(ones.shape))
    prm = P(iterations=1, beta=0.0, t=1e-300, U=1e300, lambda0=1.0, a=0.0, precond=0)
    f = np.ones((1, n, n))
    for _ in range(5):
        f, _ = oracle.reconstruct(g, counts, gamma, prm, f)
        assert abs(np.vdot(sens_img, f) - counts.sum()) < 1e-12 * counts.sum()


@pytest.mark.parametrize("kind", [0, 4])
def test_tof_converges_to_lbfgsb_minimiser(kind):
    """Theorem 2 with the TOF system matrix: the iterates reach the minimiser of Phi built from
    the dense clipping matrix weighted by h_t at the pixel centres."""
    from scipy.optimize import minimize
    n, V, nb, M, T, dtau, fwhm = 8, 18, 13, 3, 5, 9.0, 14.0
    px = 4.0
    g = oracle.geom(n, 1, V, nb, M, pixel_mm=px, sens=50.0, tof_bins=T, tof_bin_mm=dtau,
                    tof_fwhm_mm=fwhm)
    A0 = dense_A(n, V, nb) * g.sens * px
    dirs = _dirs(V)
    X = (np.arange(n) + 0.5 - n / 2.0)[None, :].repeat(n, 0).ravel()
    Y = (np.arange(n) + 0.5 - n / 2.0)[:, None].repeat(n, 1).ravel()
    rows = []
    for v in range(V):
        c, s = dirs[v]
        tau = (-X * s + Y * c) * px
        W = np.array([[h_ref(T, dtau, fwhm, t, tj) for tj in tau] for t in range(T)])
        for b in range(nb):
            for t in range(T):
                rows.append(A0[v * nb + b] * W[t])
    A = np.array(rows)                                            # [(v, b, t)][j]
    rng = np.random.default_rng(2)
    lam = A @ rng.uniform(0.5, 2.0, n * n)
    gamma = np.full((1, V, nb, T), 0.1 * lam.mean(), np.float32)
    counts = rng.poisson(lam + 0.1 * lam.mean()).astype(np.int32).reshape(1, V, nb, T)
    cnt, gam = counts.ravel().astype(float), gamma.ravel().astype(float)
    beta, gr, eps = 5.0, 2.0, 1e-12
    pairs = [(iy * n + ix, y * n + x) for iy in range(n) for ix in range(n)
             for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx or dy)
             for y, x in [(iy + dy, ix + dx)] if 0 <= y < n and 0 <= x < n]
    J, K = np.array(pairs).T

    def phi(f):
        y = A @ f
        d = f[J] - f[K]
        den = f[J] + f[K] + gr * np.abs(d) + eps
        val = y.sum() - np.dot(cnt, np.log(y + gam)) + beta * np.sum(d * d / den)
        gd = A.T @ (1 - cnt / (y + gam))
        t_ = 2 * d / den - d * d * (1 + gr * np.sign(d)) / den ** 2
        u_ = -2 * d / den - d * d * (1 - gr * np.sign(d)) / den ** 2
        gr_ = np.zeros_like(f)
        np.add.at(gr_, J, t_)
        np.add.at(gr_, K, u_)
        return val, gd + beta * gr_

    res = minimize(phi, np.ones(n * n), jac=True, method="L-BFGS-B",
                   bounds=[(0, 1000)] * (n * n), options=dict(maxiter=20000, ftol=1e-15, gtol=1e-12))
    fstar = res.x
    assert fstar.min() > 0.1
    o = oracle.objective(g, counts, gamma, fstar.reshape(1, n, n), beta)
    assert abs(o["phi"] - res.fun) < 1e-12 * abs(res.fun)
    if kind == 0:
        prm = P(iterations=400, precond=0, a=1 / 35, beta=beta)
    else:
        prm = P(iterations=400, precond=kind, a=1 / 35, rho=4.0, delta1=3.0, delta2=3.0,
                nu1=0.8, nu2=1.8, beta=beta, J1=300)
    f, _ = oracle.reconstruct(g, counts, gamma, prm, np.ones((1, n, n)))
    rel = np.linalg.norm(f.ravel() - fstar) / np.linalg.norm(fstar)
    assert rel < 5e-3, rel
