"""Pins of the oracle's fully 3-D prior (no GPU): RDP over the 26 neighbours of each voxel of a
volume (Eq. RDP and Eq. gradRD with a 3-D neighbourhood, as for the paper's fully 3-D clinical
reconstructions of Sec. IV-C), the third component of Matlab's gradient, and the 3-D
smoothness map nu (Sec. III).

Checked against: finite differences, closed forms of the 26-neighbourhood (alternating planes,
volumes constant along the planes, single planes), exact gradients of polynomials, and the
minimiser of the 3-D objective found by a general-purpose optimiser on a tiny volume.
"""
import numpy as np
import pytest

import oracle
from test_oracle_pins import dense_A


def test_rdp3d_gradient_finite_differences():
    rng = np.random.default_rng(5)
    f = rng.uniform(0.2, 3.0, (4, 6, 6))
    g = oracle.rdp_grad(f, 2.0, 1e-12, three_d=True)
    for idx in [(0, 0, 0), (1, 2, 3), (3, 5, 5), (2, 0, 4), (3, 3, 0)]:
        h = 1e-6 * f[idx]
        fp, fm = f.copy(), f.copy()
        fp[idx] += h
        fm[idx] -= h
        fd = (oracle.rdp_value(fp, 2.0, 1e-12, True) - oracle.rdp_value(fm, 2.0, 1e-12, True)) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(g[idx])), (idx, fd, g[idx])


def test_rdp3d_alternating_planes_closed_form():
    """Planes alternating a, b: only the 9 neighbours in each adjacent plane differ.  Over an
    N x N plane the neighbours a voxel has in the next plane number (3N - 2)^2 in total, so
    R = 2 (P - 1) (3N - 2)^2 (a - b)^2 / (a + b + gamma |a - b| + eps); an interior voxel has
    18 differing neighbours."""
    N, P, a, b, gr, eps = 7, 5, 1.5, 0.25, 2.0, 1e-12
    f = np.empty((P, N, N))
    for p in range(P):
        f[p] = a if p % 2 == 0 else b
    d = a - b
    den = a + b + gr * abs(d) + eps
    R = oracle.rdp_value(f, gr, eps, three_d=True)
    assert R == pytest.approx(2 * (P - 1) * (3 * N - 2) ** 2 * d * d / den, rel=1e-13)
    g = oracle.rdp_grad(f, gr, eps, three_d=True)
    # interior voxel of an a-plane: 18 neighbours of value b (Eq. gradRD's pair term)
    term = d * (gr * abs(d) + a + 3 * b + 2 * eps) / den ** 2
    assert g[2, 3, 3] == pytest.approx(2 * 18 * term, rel=1e-13)


def test_rdp3d_reduces_to_in_plane():
    """A single plane has no neighbours above or below: the 3-D prior is the in-plane one.  A
    volume constant along the planes: every in-plane offset appears at dz = -1, 0, +1 (twice on
    the first and last plane) with the same value, and the straight-up neighbours add nothing,
    so R = (3P - 2) R_plane and the gradient is 3 (2 on the end planes) times the in-plane one."""
    rng = np.random.default_rng(6)
    plane = rng.uniform(0.3, 2.0, (1, 9, 9))
    assert oracle.rdp_value(plane, three_d=True) == pytest.approx(oracle.rdp_value(plane), rel=1e-15)
    np.testing.assert_allclose(oracle.rdp_grad(plane, three_d=True), oracle.rdp_grad(plane),
                               rtol=1e-15, atol=0)
    P = 4
    vol = np.repeat(plane, P, axis=0)
    assert oracle.rdp_value(vol, three_d=True) == pytest.approx((3 * P - 2) * oracle.rdp_value(plane), rel=1e-13)
    g3 = oracle.rdp_grad(vol, three_d=True)
    g2 = oracle.rdp_grad(plane)[0]
    for p, k in enumerate([2, 3, 3, 2]):
        np.testing.assert_allclose(g3[p], k * g2, rtol=1e-12, atol=1e-15)


def test_matlab_gradient_z_exact_for_polynomials():
    """Third component of Matlab's gradient: exact for a linear function everywhere (one-sided
    differences included); for f = z^2, 2z inside, 1 on the first plane and 2P - 3 on the
    last."""
    P, N = 6, 5
    z, y, x = np.meshgrid(np.arange(P), np.arange(N), np.arange(N), indexing="ij")
    lin = 0.5 + 0.25 * x - 0.75 * y + 1.5 * z
    np.testing.assert_allclose(oracle.matlab_gradient_z(lin), 1.5, rtol=0, atol=1e-14)
    gx, gy = oracle.matlab_gradient(lin)
    np.testing.assert_allclose(gx, 0.25, atol=1e-14)
    np.testing.assert_allclose(gy, -0.75, atol=1e-14)
    gz = oracle.matlab_gradient_z(z.astype(float) ** 2)
    want = [1.0] + [2.0 * p for p in range(1, P - 1)] + [2.0 * P - 3.0]
    for p in range(P):
        np.testing.assert_array_equal(gz[p], want[p])
    assert np.all(oracle.matlab_gradient_z(np.ones((1, 3, 3))) == 0)


def test_nu3d_special_cases():
    """3-D nu (Sec. III with the volume's gradient): a ramp along the planes has uniform mu,
    hence nu = 1; a volume constant along the planes has gz = 0 and the in-plane nu."""
    ramp = (1.0 + 0.2 * np.arange(5))[:, None, None] * np.ones((5, 8, 8))
    np.testing.assert_allclose(oracle.nu_from_image(ramp, 0.5, 2.0, three_d=True), 1.0, atol=1e-14)
    rng = np.random.default_rng(8)
    vol = np.repeat(rng.uniform(0.5, 2.0, (1, 8, 8)), 3, axis=0)
    np.testing.assert_array_equal(oracle.nu_from_image(vol, 0.6, 1.8, three_d=True),
                                  oracle.nu_from_image(vol, 0.6, 1.8))
    # a step between planes: nu < 1 on the step, > 1 away from it
    step = np.ones((6, 8, 8))
    step[3:] = 3.0
    nu = oracle.nu_from_image(step, 0.5, 4.0, three_d=True)
    assert nu[2:4].max() < 1.0 and nu[0].min() > 1.0


class P:
    def __init__(self, **kw):
        d = dict(iterations=5, beta=0.05, gamma_r=2.0, eps=1e-12, t=1e-4, U=1000.0,
                 lambda0=1.0, a=0.2, rho=5.0, delta1=5.0, delta2=5.0, nu1=0.8, nu2=2.2,
                 J0=3, J1=1000, precond=4, rdp3d=1)
        d.update(kw)
        self.__dict__.update(d)


@pytest.mark.parametrize("kind", [0, 4])
def test_3d_prior_converges_to_lbfgsb_minimiser(kind):
    """Theorem 2 with the 3-D prior: the loop reaches the minimiser of Phi with R over the 26
    neighbours, found by scipy L-BFGS-B from a dense per-plane clipping matrix and an
    independently written 3-D pair list."""
    from scipy.optimize import minimize
    n, Pl, V, nb, M = 6, 3, 18, 11, 3
    g = oracle.geom(n, Pl, V, nb, M, pixel_mm=4.0, sens=50.0)
    A1 = dense_A(n, V, nb) * g.sens * g.pixel_mm
    rng = np.random.default_rng(3)
    truth = rng.uniform(0.5, 2.0, (Pl, n * n))
    lam = np.stack([A1 @ truth[p] for p in range(Pl)])
    gamma = np.full((Pl, V, nb), 0.1 * lam.mean(), np.float32)
    counts = rng.poisson(lam.reshape(Pl, V, nb) + gamma).astype(np.int32)
    cnt, gam = counts.reshape(Pl, -1).astype(float), gamma.reshape(Pl, -1).astype(float)
    beta, gr, eps = 5.0, 2.0, 1e-12
    idx = lambda p, y, x: (p * n + y) * n + x
    pairs = [(idx(p, y, x), idx(p + dz, y + dy, x + dx))
             for p in range(Pl) for y in range(n) for x in range(n)
             for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
             if (dx or dy or dz) and 0 <= p + dz < Pl and 0 <= y + dy < n and 0 <= x + dx < n]
    J, K = np.array(pairs).T

    def phi(fv):
        f = fv.reshape(Pl, n * n)
        y = np.stack([A1 @ f[p] for p in range(Pl)])
        d = fv[J] - fv[K]
        den = fv[J] + fv[K] + gr * np.abs(d) + eps
        val = y.sum() - np.sum(cnt * np.log(y + gam)) + beta * np.sum(d * d / den)
        gd = np.stack([A1.T @ (1 - cnt[p] / (y[p] + gam[p])) for p in range(Pl)]).ravel()
        t = 2 * d / den - d * d * (1 + gr * np.sign(d)) / den ** 2
        u = -2 * d / den - d * d * (1 - gr * np.sign(d)) / den ** 2
        gr_ = np.zeros_like(fv)
        np.add.at(gr_, J, t)
        np.add.at(gr_, K, u)
        return val, gd + beta * gr_

    res = minimize(phi, np.ones(Pl * n * n), jac=True, method="L-BFGS-B",
                   bounds=[(0, 1000)] * (Pl * n * n),
                   options=dict(maxiter=20000, ftol=1e-15, gtol=1e-12))
    fstar = res.x
    assert fstar.min() > 0.1
    o = oracle.objective(g, counts, gamma, fstar.reshape(Pl, n, n), beta, three_d=True)
    assert abs(o["phi"] - res.fun) < 1e-12 * abs(res.fun)
    if kind == 0:
        prm = P(iterations=400, precond=0, a=1 / 35, beta=beta)
    else:
        prm = P(iterations=400, precond=4, a=1 / 35, rho=4.0, delta1=3.0, delta2=3.0,
                nu1=0.8, nu2=1.8, beta=beta, J1=300)
    f, _ = oracle.reconstruct(g, counts, gamma, prm, np.ones((Pl, n, n)))
    rel = np.linalg.norm(f.ravel() - fstar) / np.linalg.norm(fstar)
    assert rel < 5e-3, rel
    # and the in-plane prior has another minimiser: the 3-D neighbourhood is in effect
    f2, _ = oracle.reconstruct(g, counts, gamma, P(**{**prm.__dict__, "rdp3d": 0}), np.ones((Pl, n, n)))
    assert np.linalg.norm(f2.ravel() - fstar) / np.linalg.norm(fstar) > 2 * rel
