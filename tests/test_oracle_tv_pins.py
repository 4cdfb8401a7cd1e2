"""Pins of the oracle's TV variant (no GPU).

The paper's prior is RDP, handled by its gradient; the TV variant puts total variation into the
same preconditioned step through a proximal step in the step sizes' metric,
x = argmin 1/2 sum (x - z)^2 / W + b R_TV(x), approximated by primal-dual (Chambolle-Pock)
iterations.  Checked against: closed forms of R_TV, the closed-form weighted proximal step of a
two-column image, the duality gap of the primal-dual pair (weak duality certifies optimality),
b = 0, and the minimiser of F + beta R_TV found by a general-purpose optimiser.
"""
import numpy as np
import pytest

import oracle
from test_oracle_pins import dense_A


def test_tv_value_closed_forms():
    N = 9
    assert oracle.tv_value(np.full((2, N, N), 3.0)) == 0.0
    edge = np.ones((1, N, N))
    edge[0, :, 4:] = 2.5                      # one jump of 1.5 per row, across columns 3 -> 4
    assert oracle.tv_value(edge) == pytest.approx(N * 1.5, rel=1e-15)
    ramp = np.tile(0.7 * np.arange(N), (N, 1))[None]      # gx = 0.7 except at the last column
    assert oracle.tv_value(ramp) == pytest.approx(N * (N - 1) * 0.7, rel=1e-14)
    diag = np.add.outer(np.arange(N), np.arange(N))[None] * 1.0   # gx = gy = 1 inside
    want = (N - 1) ** 2 * np.sqrt(2.0) + 2 * (N - 1)             # last row / column: one component
    assert oracle.tv_value(diag) == pytest.approx(want, rel=1e-14)


def _prox_two_columns(z1, z2, w1, w2, b):
    """argmin 1/2 ((x1 - z1)^2 / w1 + (x2 - z2)^2 / w2) + b |x2 - x1| (closed form)."""
    d = z2 - z1
    if abs(d) <= b * (w1 + w2):
        m = (z1 / w1 + z2 / w2) / (1 / w1 + 1 / w2)
        return m, m
    s = np.sign(d)
    return z1 + s * b * w1, z2 - s * b * w2


@pytest.mark.parametrize("z1,z2,w1,w2,b", [(1.0, 3.0, 0.5, 2.0, 0.2), (1.0, 1.4, 0.5, 2.0, 0.3),
                                           (2.0, -1.0, 1.5, 0.25, 0.4)])
def test_tv_prox_two_columns(z1, z2, w1, w2, b):
    """Two identical rows: the isotropic TV is |x2 - x1| per row and the weighted proximal step
    has a closed form (soft threshold of the difference, or the W^-1-weighted mean)."""
    z = np.array([[[z1, z2], [z1, z2]]])
    W = np.array([[[w1, w2], [w1, w2]]])
    x, (px, py) = oracle.tv_prox(z, W, b, 4000)
    x1, x2 = _prox_two_columns(z1, z2, w1, w2, b)
    np.testing.assert_allclose(x[0], [[x1, x2], [x1, x2]], rtol=0, atol=1e-10)
    assert np.all(np.hypot(px, py) <= 1 + 1e-15)


def test_tv_prox_duality_gap():
    """Weak duality: P(x) = 1/2 ||x - z||^2_{W^-1} + b R_TV(x) >= D(p) = <z, K^T p> -
    1/2 ||K^T p||^2_W for every |p_j| <= 1, K^T p = -b div p; the gap of the iterates vanishes,
    which certifies the proximal point without another solver."""
    rng = np.random.default_rng(4)
    z = rng.uniform(-1.0, 3.0, (2, 8, 8))
    W = rng.uniform(0.5, 2.0, (2, 8, 8))
    b = 0.3
    x, (px, py) = oracle.tv_prox(z, W, b, 20000)
    primal = 0.5 * np.sum((x - z) ** 2 / W) + b * oracle.tv_value(x)
    div = px.copy()
    div[:, :, 1:] -= px[:, :, :-1]
    div += py
    div[:, 1:, :] -= py[:, :-1, :]
    kt = -b * div
    dual = np.sum(z * kt) - 0.5 * np.sum(W * kt * kt)
    assert np.all(np.hypot(px, py) <= 1 + 1e-15)
    assert -1e-12 <= primal - dual <= 1e-9 * abs(primal), (primal, dual)
    # too few iterations leave a visible gap: the certificate is not vacuous
    x5, (p5x, p5y) = oracle.tv_prox(z, W, b, 5)
    d5 = p5x.copy()
    d5[:, :, 1:] -= p5x[:, :, :-1]
    d5 += p5y
    d5[:, 1:, :] -= p5y[:, :-1, :]
    k5 = -b * d5
    gap5 = 0.5 * np.sum((x5 - z) ** 2 / W) + b * oracle.tv_value(x5) - (np.sum(z * k5) - 0.5 * np.sum(W * k5 * k5))
    assert gap5 > 1e-4


def test_tv_prox_zero_weight_is_identity():
    z = np.random.default_rng(2).uniform(0, 1, (1, 6, 6))
    x, _ = oracle.tv_prox(z, np.ones_like(z), 0.0, 50)
    np.testing.assert_array_equal(x, z)


class P:
    def __init__(self, **kw):
        d = dict(iterations=3, beta=0.0, gamma_r=2.0, eps=1e-12, t=1e-4, U=1000.0,
                 lambda0=1.0, a=0.2, rho=2.0, delta1=5.0, delta2=5.0, nu1=0.8, nu2=1.5,
                 J0=3, J1=1000, precond=4, rdp3d=0, reg=1, tv_iters=10)
        d.update(kw)
        self.__dict__.update(d)


def test_tv_loop_without_penalty_is_the_rdp_loop_without_penalty():
    from paper_2111_07886_gb300 import synth
    w = synth.Workload("t", 16, 2, 4.0, 24, 23, 4.0, 4, 4e4, "ellipsoid3d", synth.AlgoParams(),
                       plane_mm=4.0, seed=3)
    scan = synth.make_scan(w)
    g = oracle.geom(16, 2, 24, 23, 4, pixel_mm=4.0, sens=scan["sens"])
    f0 = np.ones((2, 16, 16))
    a, _ = oracle.reconstruct(g, scan["counts"], scan["gamma"], P(reg=1), f0)
    b, _ = oracle.reconstruct(g, scan["counts"], scan["gamma"], P(reg=0), f0)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=0)


def test_tv_loop_converges_to_minimiser():
    """The TV variant of the loop (BSREM schedule, 40 primal-dual iterations per step, warm
    dual) approaches the minimiser of F + beta R_TV on the box: scipy L-BFGS-B on the TV smoothed
    by sqrt(|Df|^2 + 1e-12), from a dense clipping matrix; the smoothing moves Phi by at most
    beta * 1e-6 * (number of voxels)."""
    from scipy.optimize import minimize
    n, V, nb, M = 8, 24, 15, 3
    g = oracle.geom(n, 1, V, nb, M, pixel_mm=4.0, sens=50.0)
    A = dense_A(n, V, nb) * g.sens * g.pixel_mm
    rng = np.random.default_rng(0)
    truth = np.ones((n, n))
    truth[2:6, 3:7] = 2.5
    lam = A @ truth.ravel()
    gamma = np.full((1, V, nb), 0.1 * lam.mean(), np.float32)
    counts = rng.poisson(lam + 0.1 * lam.mean()).astype(np.int32).reshape(1, V, nb)
    cnt, gam = counts.ravel().astype(float), gamma.ravel().astype(float)
    beta, e2 = 20.0, 1e-12

    def grad_ops(f):
        F = f.reshape(n, n)
        gx = np.zeros_like(F)
        gy = np.zeros_like(F)
        gx[:, :-1] = F[:, 1:] - F[:, :-1]
        gy[:-1, :] = F[1:, :] - F[:-1, :]
        return gx, gy

    def phi(f):
        y = A @ f
        gx, gy = grad_ops(f)
        nrm = np.sqrt(gx * gx + gy * gy + e2)
        val = y.sum() - np.dot(cnt, np.log(y + gam)) + beta * nrm.sum()
        ux, uy = gx / nrm, gy / nrm
        gtv = np.zeros((n, n))                # D^T u = -div u
        gtv[:, :-1] -= ux[:, :-1]
        gtv[:, 1:] += ux[:, :-1]
        gtv[:-1, :] -= uy[:-1, :]
        gtv[1:, :] += uy[:-1, :]
        return val, A.T @ (1 - cnt / (y + gam)) + beta * gtv.ravel()

    res = minimize(phi, np.ones(n * n), jac=True, method="L-BFGS-B", bounds=[(1e-6, 1000)] * (n * n),
                   options=dict(maxiter=50000, ftol=1e-16, gtol=1e-12))
    fstar = res.x
    prm = P(iterations=300, precond=0, a=1 / 35, beta=beta, tv_iters=40)
    f, obj = oracle.reconstruct(g, counts, gamma, prm, np.ones((1, n, n)), with_objective=True)
    o_f = oracle.objective(g, counts, gamma, f, beta, tv=True)["phi"]
    o_s = oracle.objective(g, counts, gamma, fstar.reshape(1, n, n), beta, tv=True)["phi"]
    assert o_f <= o_s + 1e-6 * abs(o_s), (o_f, o_s)
    rel = np.linalg.norm(f.ravel() - fstar) / np.linalg.norm(fstar)
    assert rel < 1e-2, rel
    assert obj[-1] < obj[0]
