"""Pins of the oracle's per-bin detection factors (no GPU): the system matrix diag(a) A of a
scan with attenuation (the simulated system of Sec. IV-A includes uniform water attenuation).

Checked against: the plain model when a = 1 (bitwise); a constant factor c, which is the plain
model with sens scaled by c; Shepp-Vardi EM count preservation with sum_j (A^T a)_j f_j (Sec. I)
for random a; p_j of Eq. pj from a dense clipping matrix with different factors per plane; and
L-BFGS-B on Phi built from the dense matrix diag(a) A (Theorem 2: the iteration converges to
its minimiser), none of which uses the oracle's projector.
"""
import numpy as np
import pytest

import oracle
from test_oracle_pins import P, _small_problem, dense_A


def _two_plane_problem(n=16, V=24, nb=23, M=4, seed=11):
    from paper_2111_07886_gb300 import synth
    w = synth.Workload("t", n, 2, 4.0, V, nb, 4.0, M, 4e4, "ellipsoid3d", synth.AlgoParams(),
                       plane_mm=4.0, seed=seed)
    scan = synth.make_scan(w)
    return oracle.geom(n, 2, V, nb, M, pixel_mm=4.0, bin_mm=4.0, sens=scan["sens"]), scan


def _factors(shape, seed, lo=0.2, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, shape).astype(np.float32)


def test_unit_factors_are_the_plain_model():
    g, scan = _two_plane_problem()
    ones = np.ones(scan["counts"].shape, np.float32)
    f0 = np.ones((2, g.n, g.n))
    for kw in (dict(), dict(precond=0), dict(precond=3, J0=1)):
        a, oa = oracle.reconstruct(g, scan["counts"], scan["gamma"], P(iterations=3, **kw), f0,
                                   with_objective=True)
        b, ob = oracle.reconstruct(g, scan["counts"], scan["gamma"], P(iterations=3, **kw), f0,
                                   with_objective=True, mult=ones)
        np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(oa, ob)
    p2 = oracle.sensitivity_m(g, ones)
    np.testing.assert_array_equal(p2, np.stack([oracle.sensitivity(g)] * 2))


@pytest.mark.parametrize("c", [0.375, 2.5])
def test_constant_factor_is_a_sensitivity_scale(c):
    """a_i = c for every bin is A scaled by c: the same iterates and objective as the plain model
    with sens c times larger (beta > 0, so p enters the step through the prior term too), up to
    rounding; c is exact in float32 and the P2 settings are the well-conditioned ones."""
    g, scan = _small_problem(M=4)
    f0 = np.ones((1, g.n, g.n))
    gc = oracle.geom(g.n, 1, g.nviews, g.nbins, g.nsubsets, g.pixel_mm, g.bin_mm, g.sens * c)
    mult = np.full(scan["counts"].shape, c, np.float32)
    prm = P(iterations=4, beta=0.5, a=0.45, rho=2.0, nu2=1.5, J0=2)
    a, oa = oracle.reconstruct(gc, scan["counts"], scan["gamma"], prm, f0, with_objective=True)
    b, ob = oracle.reconstruct(g, scan["counts"], scan["gamma"], prm, f0, with_objective=True,
                               mult=mult)
    assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(a), np.linalg.norm(a - b) / np.linalg.norm(a)
    np.testing.assert_allclose(ob, oa, rtol=1e-12)
    np.testing.assert_allclose(oracle.sensitivity_m(g, mult)[0], c * oracle.sensitivity(g),
                               rtol=1e-12)


def test_em_count_preservation_with_factors():
    """M = 1, beta = 0, gamma -> 0, lambda = alpha = nu = 1: the step is EM for diag(a) A,
    f <- f (A^T a(g / (a A f))) / A^T a, so sum_j (A^T a)_j f_j = sum_i g_i every iteration."""
    n, V, nb = 16, 20, 25
    g = oracle.geom(n, 2, V, nb, 1, pixel_mm=2.0, sens=3.0)
    rng = np.random.default_rng(5)
    ones_proj = oracle.forward(g, -1, np.ones((2, n, n)))
    hit = ones_proj > 0
    counts = np.where(hit, rng.integers(1, 50, ones_proj.shape), 0).astype(np.int32)
    gamma = np.full(ones_proj.shape, 1e-30, np.float32)
    mult = _factors(ones_proj.shape, 9)
    sens_img = oracle.back(g, -1, mult.astype(np.float64))
    prm = P(iterations=1, beta=0.0, t=1e-300, U=1e300, lambda0=1.0, a=0.0, precond=0)
    f = np.ones((2, n, n))
    for _ in range(6):
        f, _ = oracle.reconstruct(g, counts, gamma, prm, f, mult=mult)
        assert abs(np.vdot(sens_img, f) - counts.sum()) < 1e-12 * counts.sum()
    # without the factors in the model the same data are not preserved
    f1, _ = oracle.reconstruct(g, counts, gamma, prm, np.ones((2, n, n)))
    assert abs(np.vdot(sens_img, f1) - counts.sum()) > 1e-3 * counts.sum()


def test_sensitivity_per_voxel_from_dense_matrix():
    """p_j = (A^T a)_j / M per plane (Eq. pj with the factors in A), from the clipping matrix."""
    n, V, nb, M, Pn = 8, 9, 13, 3, 3
    g = oracle.geom(n, Pn, V, nb, M, pixel_mm=1.0, sens=1.7)
    A = dense_A(n, V, nb) * g.sens * g.pixel_mm
    mult = _factors((Pn, V, nb), 4)
    mult[1, :, : nb // 2] = 1.0
    got = oracle.sensitivity_m(g, mult)
    for p in range(Pn):
        col = A.T @ mult[p].astype(np.float64).ravel()
        want = np.where(col > 0, col / M, 1.0 / M)
        np.testing.assert_allclose(got[p].ravel(), want, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("kind", [0, 4])
def test_converges_to_lbfgsb_minimiser_with_factors(kind):
    """Theorem 2 for diag(a) A: the oracle's iterates reach the minimiser of
    Phi(f) = sum(a A f) - sum g ln(a A f + gamma) + beta R(f) found by scipy L-BFGS-B on the
    dense clipping matrix; the oracle's Phi equals the independent Phi there."""
    from scipy.optimize import minimize
    n, V, nb, M = 8, 24, 15, 3
    g = oracle.geom(n, 1, V, nb, M, pixel_mm=4.0, sens=50.0)
    mult = _factors((1, V, nb), 21, lo=0.3, hi=1.0)
    A = dense_A(n, V, nb) * g.sens * g.pixel_mm * mult.astype(np.float64).reshape(-1, 1)
    rng = np.random.default_rng(1)
    lam = A @ rng.uniform(0.5, 2.0, n * n)
    gamma = np.full((1, V, nb), 0.1 * lam.mean(), np.float32)
    counts = rng.poisson(lam + 0.1 * lam.mean()).astype(np.int32).reshape(1, V, nb)
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
        t = 2 * d / den - d * d * (1 + gr * np.sign(d)) / den ** 2
        u = -2 * d / den - d * d * (1 - gr * np.sign(d)) / den ** 2
        gr_ = np.zeros_like(f)
        np.add.at(gr_, J, t)
        np.add.at(gr_, K, u)
        return val, gd + beta * gr_

    res = minimize(phi, np.ones(n * n), jac=True, method="L-BFGS-B",
                   bounds=[(0, 1000)] * (n * n), options=dict(maxiter=20000, ftol=1e-15, gtol=1e-12))
    fstar = res.x
    assert fstar.min() > 0.1
    o = oracle.objective(g, counts, gamma, fstar.reshape(1, n, n), beta, mult=mult)
    assert abs(o["phi"] - res.fun) < 1e-12 * abs(res.fun)
    if kind == 0:
        prm = P(iterations=400, precond=0, a=1 / 35, beta=beta)
    else:
        prm = P(iterations=400, precond=kind, a=1 / 35, rho=4.0, delta1=3.0, delta2=3.0,
                nu1=0.8, nu2=1.8, beta=beta, J1=300)
    f, _ = oracle.reconstruct(g, counts, gamma, prm, np.ones((1, n, n)), mult=mult)
    rel = np.linalg.norm(f.ravel() - fstar) / np.linalg.norm(fstar)
    assert rel < 5e-3, rel
    # the plain model on the same data converges elsewhere
    f0, _ = oracle.reconstruct(g, counts, gamma, prm, np.ones((1, n, n)))
    assert np.linalg.norm(f0.ravel() - fstar) / np.linalg.norm(fstar) > 5e-2
