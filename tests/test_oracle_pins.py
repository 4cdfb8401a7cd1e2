"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a dense system matrix
built by clipping every ray against every pixel square, closed-form line integrals,
finite differences, invariants of the method (Sec. II-III, App. A-B), the textbook EM
special case, and a general-purpose optimiser reaching the same minimiser.
"""
import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------------------------------------
# Dense brute-force system matrix: clip the line {X c + Y s = r} against each pixel
# square (Liang-Barsky in the line parameter tau), half-open pixels [x, x+1) x [y, y+1).
# ------------------------------------------------------------------------------------
def _dirs(nviews):
    out = []
    for v in range(nviews):
        th = v * math.pi / nviews
        c, s = math.cos(th), math.sin(th)
        if abs(c) < 1e-12:
            c, s = 0.0, math.copysign(1.0, s)
        if abs(s) < 1e-12:
            s, c = 0.0, math.copysign(1.0, c)
        out.append((c, s))
    return out


def dense_A(n, nviews, nbins, rho=1.0, views=None):
    """Rows (v, b) for v in `views`; columns = flat pixel index; lengths in pixel units."""
    views = list(range(nviews)) if views is None else views
    dirs = _dirs(nviews)
    x0 = (np.arange(n) - n / 2.0)[None, :].repeat(n, 0).ravel()   # column ix -> X lower edge
    y0 = (np.arange(n) - n / 2.0)[:, None].repeat(n, 1).ravel()   # row iy -> Y lower edge
    A = np.zeros((len(views) * nbins, n * n))
    for u, v in enumerate(views):
        c, s = dirs[v]
        for b in range(nbins):
            r = (b - (nbins - 1) / 2.0) * rho
            lo = np.full(n * n, -np.inf)
            hi = np.full(n * n, np.inf)
            ok = np.ones(n * n, bool)
            # X(tau) = r c - tau s in [x0, x0 + 1]
            if s == 0.0:
                X = r * c
                ok &= (x0 <= X) & (X < x0 + 1)
            else:
                t1, t2 = (r * c - x0) / s, (r * c - x0 - 1) / s
                lo = np.maximum(lo, np.minimum(t1, t2))
                hi = np.minimum(hi, np.maximum(t1, t2))
            # Y(tau) = r s + tau c in [y0, y0 + 1]
            if c == 0.0:
                Y = r * s
                ok &= (y0 <= Y) & (Y < y0 + 1)
            else:
                t1, t2 = (y0 - r * s) / c, (y0 + 1 - r * s) / c
                lo = np.maximum(lo, np.minimum(t1, t2))
                hi = np.minimum(hi, np.maximum(t1, t2))
            A[u * nbins + b] = np.where(ok, np.clip(hi - lo, 0.0, None), 0.0)
    return A


@pytest.mark.parametrize("n,nviews,nbins,rho", [(8, 8, 11, 1.0), (8, 7, 12, 1.0),
                                                (8, 12, 15, 0.7), (16, 16, 23, 1.0),
                                                (16, 9, 17, 1.3)])
def test_siddon_matches_dense_bruteforce(n, nviews, nbins, rho):
    """Oracle Siddon rows == dense clipping rows to 1e-12 (the ray-driven model of Sec. IV-A,
    one line per bin)."""
    g = oracle.geom(n, 1, nviews, nbins, 1, pixel_mm=1.0, bin_mm=rho)
    A = dense_A(n, nviews, nbins, rho)
    for v in range(nviews):
        for b in range(nbins):
            pix, ln = oracle.ray_pieces(g, v, b)
            row = np.zeros(n * n)
            np.add.at(row, pix, ln)
            np.testing.assert_allclose(row, A[v * nbins + b], rtol=0, atol=1e-12)


def test_forward_equals_dense_matrix_per_subset():
    """ora_forward over every unit image reproduces sens * pixel_mm * dense A_i (Sec. II-B)."""
    n, V, nb, M = 8, 12, 13, 3
    pixel_mm, sens = 2.5, 0.37
    g = oracle.geom(n, 1, V, nb, M, pixel_mm=pixel_mm, bin_mm=pixel_mm, sens=sens)
    for i in range(M):
        views = list(range(i, V, M))
        A = dense_A(n, V, nb, 1.0, views) * sens * pixel_mm
        cols = np.zeros_like(A)
        for j in range(n * n):
            e = np.zeros((1, n, n))
            e.flat[j] = 1.0
            cols[:, j] = oracle.forward(g, i, e).ravel()
        np.testing.assert_allclose(cols, A, rtol=0, atol=1e-12)


def test_adjointness_every_subset():
    """<A_i x, y> = <x, A_i^T y> to 1e-12 relative for random x, y and every subset."""
    n, P, V, nb, M = 24, 3, 30, 35, 5
    g = oracle.geom(n, P, V, nb, M, pixel_mm=1.7, bin_mm=1.7, sens=2.0)
    rng = np.random.default_rng(1)
    for i in range(M):
        x = rng.uniform(0, 1, (P, n, n))
        y = rng.uniform(0, 1, (P, oracle.subset_size(g, i), nb))
        lhs = np.vdot(oracle.forward(g, i, x), y)
        rhs = np.vdot(x, oracle.back(g, i, y))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _square_chord(n, c, s, r):
    """Length of the line {Xc + Ys = r} inside the half-open square [-n/2, n/2)^2."""
    h = n / 2.0
    lo, hi = -np.inf, np.inf
    if s == 0.0:
        if not (-h <= r * c < h):
            return 0.0
    else:
        t1, t2 = (r * c + h) / s, (r * c - h) / s
        lo, hi = max(lo, min(t1, t2)), min(hi, max(t1, t2))
    if c == 0.0:
        if not (-h <= r * s < h):
            return 0.0
    else:
        t1, t2 = (-h - r * s) / c, (h - r * s) / c
        lo, hi = max(lo, min(t1, t2)), min(hi, max(t1, t2))
    return max(0.0, hi - lo)


def test_all_ones_image_gives_square_chord():
    """All-ones image: each projection is the chord of the line through the FOV square."""
    n, V, nb = 32, 36, 47
    g = oracle.geom(n, 1, V, nb, 1)
    y = oracle.forward(g, -1, np.ones((1, n, n)))[0]
    for v, (c, s) in enumerate(_dirs(V)):
        for b in range(nb):
            r = b - (nb - 1) / 2.0
            assert abs(y[v, b] - _square_chord(n, c, s, r)) < 1e-11


def test_single_pixel_trapezoid_profile():
    """Single hot pixel: the projection of a unit square is the trapezoid
    min(1/a, max(0, ((a+b)/2 - |d|) / (a b))), a = max(|c|,|s|), b = min(|c|,|s|); for b = 0
    the half-open rule gives 1 for d in [-1/2, 1/2) and 0 elsewhere."""
    n, V, nb = 16, 24, 33
    g = oracle.geom(n, 1, V, nb, 1, bin_mm=0.37)
    ix, iy = 5, 11
    f = np.zeros((1, n, n))
    f[0, iy, ix] = 1.0
    y = oracle.forward(g, -1, f)[0]
    xc, yc = ix + 0.5 - n / 2.0, iy + 0.5 - n / 2.0
    for v, (c, s) in enumerate(_dirs(V)):
        a, bb = max(abs(c), abs(s)), min(abs(c), abs(s))
        for b in range(nb):
            d = (b - (nb - 1) / 2.0) * 0.37 - (xc * c + yc * s)
            if bb == 0.0:
                want = 1.0 if -0.5 <= d < 0.5 else 0.0
            else:
                want = min(1.0 / a, max(0.0, ((a + bb) / 2 - abs(d)) / (a * bb)))
            assert abs(y[v, b] - want) < 1e-12, (v, b, y[v, b], want)


def test_uniform_disk_line_integrals():
    """Pixelised uniform disk of radius R: projections approach 2 sqrt(R^2 - s^2) (the
    continuous line integral) to within the partial-volume error of the boundary pixels:
    under 2 % for rays through the inner half of the disk (R = 40 px)."""
    n, V, nb, R = 128, 12, 129, 40.0
    ss = 8
    gpx = (np.arange(n * ss) + 0.5) / ss - n / 2.0
    X, Y = np.meshgrid(gpx, gpx)
    disk = ((X ** 2 + Y ** 2) <= R * R).reshape(n, ss, n, ss).mean(axis=(1, 3))
    g = oracle.geom(n, 1, V, nb, 1)
    y = oracle.forward(g, -1, disk[None])[0]
    r = np.arange(nb) - (nb - 1) / 2.0
    inside = np.abs(r) < 0.5 * R
    want = 2.0 * np.sqrt(np.clip(R * R - r * r, 0, None))
    rel = np.abs(y[:, inside] - want[inside]) / want[inside]
    assert rel.max() < 0.02, rel.max()
    assert np.abs(y[:, np.abs(r) > R + 1]).max() == 0.0


# ------------------------------------------------------------------------------------
# RDP (Eq. RDP) and its derivatives (App. A)
# ------------------------------------------------------------------------------------
def test_sensitivity_is_column_sums_over_M():
    """p_j = (A^T 1)_j / M, and 1/M for pixels no ray reaches (Eq. pj)."""
    n, V, nb, M = 12, 2, 5, 2           # 5 bins at 0 and pi/2 leave the corners unreached
    g = oracle.geom(n, 1, V, nb, M, pixel_mm=1.5, sens=0.6)
    col = (dense_A(n, V, nb) * g.sens * g.pixel_mm).sum(axis=0)
    assert (col == 0).any()
    want = np.where(col > 0, col / M, 1.0 / M)
    np.testing.assert_allclose(oracle.sensitivity(g).ravel(), want, rtol=1e-13, atol=1e-15)


def test_rdp_closed_forms():
    n = 6
    const = np.full((1, n, n), 3.7)
    assert oracle.rdp_value(const) == 0.0
    assert np.abs(oracle.rdp_grad(const)).max() == 0.0
    # checkerboard a/b: every ordered neighbour pair of unlike values contributes
    # (a-b)^2 / (a+b+gamma_R|a-b|+eps); unlike pairs are the 4-neighbour ones.
    a, b, gr, eps = 2.0, 0.5, 2.0, 1e-12
    iy, ix = np.mgrid[0:n, 0:n]
    f = np.where((ix + iy) % 2 == 0, a, b)[None]
    unlike_ordered = 2 * (2 * n * (n - 1))          # horizontal + vertical, both orders
    want = unlike_ordered * (a - b) ** 2 / (a + b + gr * abs(a - b) + eps)
    assert abs(oracle.rdp_value(f, gr, eps) - want) < 1e-12 * want


def test_rdp_gradient_finite_differences():
    rng = np.random.default_rng(3)
    f = rng.uniform(0.2, 3.0, (2, 9, 9))
    g = oracle.rdp_grad(f, 2.0, 1e-12)
    fd = np.zeros_like(f)
    for idx in np.ndindex(f.shape):
        h = 1e-6 * f[idx]
        fp, fm = f.copy(), f.copy()
        fp[idx] += h
        fm[idx] -= h
        fd[idx] = (oracle.rdp_value(fp) - oracle.rdp_value(fm)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8)


def _rdp_hessian_closed_form(f, gr=2.0, eps=1e-12):
    """Eq. SecondDerivative of App. A, one plane, dense."""
    n = f.shape[0]
    H = np.zeros((n * n, n * n))
    for iy in range(n):
        for ix in range(n):
            j = iy * n + ix
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dx == 0 and dy == 0:
                        continue
                    y, x = iy + dy, ix + dx
                    if not (0 <= x < n and 0 <= y < n):
                        continue
                    k = y * n + x
                    fj, fk = f[iy, ix], f[y, x]
                    den = (fj + fk + gr * abs(fj - fk) + eps) ** 3
                    H[j, j] += 4 * (2 * fk + eps) ** 2 / den
                    H[j, k] = -4 * (4 * fj * fk + 2 * eps * (fj + fk) + eps ** 2) / den
    return H


def test_rdp_hessian_fd_symmetric_psd_nullspace():
    """Finite differences of the oracle gradient give the App. A Hessian; it is symmetric,
    positive semidefinite, and x = 2f + eps is in its null space (Eq. Hessian_R).  Like
    Eq. gradRD, Eq. SecondDerivative already counts both ordered pairs (j,k) and (k,j)."""
    rng = np.random.default_rng(5)
    n = 5
    f = rng.uniform(0.5, 2.0, (n, n))
    H_fd = np.zeros((n * n, n * n))
    for j in range(n * n):
        h = 1e-6 * f.flat[j]
        fp, fm = f.copy(), f.copy()
        fp.flat[j] += h
        fm.flat[j] -= h
        H_fd[:, j] = (oracle.rdp_grad(fp[None]) - oracle.rdp_grad(fm[None])).ravel() / (2 * h)
    H = _rdp_hessian_closed_form(f)
    np.testing.assert_allclose(H_fd, H, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(H_fd, H_fd.T, rtol=1e-5, atol=1e-6)
    w = np.linalg.eigvalsh(0.5 * (H + H.T))
    assert w.min() > -1e-10 * w.max()
    x = (2 * f + 1e-12).ravel()
    assert np.abs(H @ x).max() < 1e-9 * np.abs(H).max() * np.abs(x).max()


def test_grad_F_finite_differences():
    """grad F = A^T (1 - g / (A f + gamma)) (App. A) against FD of F (Eq. FidelityTerm)."""
    n, V, nb = 10, 12, 15
    g = oracle.geom(n, 1, V, nb, 1, pixel_mm=2.0, sens=0.8)
    rng = np.random.default_rng(7)
    f = rng.uniform(0.5, 2.0, (1, n, n))
    counts = rng.poisson(5.0, (1, V, nb)).astype(np.int32)
    gamma = np.full((1, V, nb), 0.3, np.float32)
    y = oracle.forward(g, -1, f)
    gradF = oracle.back(g, -1, 1.0 - counts / (y + gamma.astype(np.float64)))

    def F(ff):
        o = oracle.objective(g, counts, gamma, ff, beta=0.0)
        return o["sum_af"] - o["sum_glog"]

    fd = np.zeros_like(f)
    for idx in np.ndindex(f.shape):
        h = 1e-5
        fp, fm = f.copy(), f.copy()
        fp[idx] += h
        fm[idx] -= h
        fd[idx] = (F(fp) - F(fm)) / (2 * h)
    np.testing.assert_allclose(gradF, fd, rtol=1e-6, atol=1e-7)


def _load_golden_gradient():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "matlab_gradient_4x4.txt"))
            if l.strip() and not l.startswith("#")]
    a = np.array(rows, dtype=float)
    return a[0:4], a[4:8], a[8:12]


def test_matlab_gradient_golden():
    F, gx, gy = _load_golden_gradient()
    ox, oy = oracle.matlab_gradient(F[None])
    np.testing.assert_array_equal(ox[0], gx)
    np.testing.assert_array_equal(oy[0], gy)


def test_nu_special_cases():
    """nu (Eq. nuki, Sec. III): a constant or linear-ramp image has uniform mu, hence
    nu = P(1) = 1; a step image gets nu < 1 on the step and > 1 in the flat parts."""
    n = 12
    np.testing.assert_allclose(oracle.nu_from_image(np.full((1, n, n), 2.0), 0.5, 2.0), 1.0, rtol=0, atol=1e-14)
    ramp = (1.0 + 0.1 * np.arange(n))[None, None, :].repeat(n, 1)
    np.testing.assert_allclose(oracle.nu_from_image(ramp, 0.5, 2.0), 1.0, rtol=0, atol=1e-14)
    step = np.ones((1, n, n))
    step[0, :, n // 2:] = 3.0
    nu = oracle.nu_from_image(step, 0.5, 4.0)[0]
    assert nu[:, n // 2].max() < 1.0 and nu[:, 0].min() > 1.0
    # clamping to [nu1, nu2]
    nu_c = oracle.nu_from_image(step, 0.9, 1.1)[0]
    assert nu_c.min() >= 0.9 and nu_c.max() <= 1.1


# ------------------------------------------------------------------------------------
# Scalar schedules (Eqs. preconditioner:Nesterov and preconditioner:KM, App. B)
# ------------------------------------------------------------------------------------
def test_alpha_nesterov_limits():
    M = 12
    K = 4000
    a = oracle.alpha_nesterov(M * K)
    assert a[0] == 1.0
    assert np.all(np.diff(a) > 0) and a[-1] < 2.0
    k = K - 1
    for i in range(M):
        lim = k * (2.0 - a[k * M + i])
        assert abs(lim - 3.0 / M) < 2e-3 * 3.0 / M, lim


def test_alpha_km_limits():
    M, rho, d1, d2 = 24, 4.0, 3.0, 3.0
    K = 100000
    a = oracle.alpha_km(M * K, rho, d1, d2)
    assert a[0] == pytest.approx(1.0, abs=1e-15)       # delta2 = delta1 => alpha_{0,1} = 1
    k = K - 1
    for i in range(M):
        lim = k * (rho - a[k * M + i])
        assert abs(lim - (rho * d1 - d2) / M) < 1e-3, lim


# ------------------------------------------------------------------------------------
# The whole loop (Table I)
# ------------------------------------------------------------------------------------
class P:
    def __init__(self, **kw):
        d = dict(iterations=5, beta=0.05, gamma_r=2.0, eps=1e-12, t=1e-4, U=1000.0,
                 lambda0=1.0, a=0.2, rho=5.0, delta1=5.0, delta2=5.0, nu1=0.8, nu2=2.2,
                 J0=3, J1=1000, precond=4)
        d.update(kw)
        self.__dict__.update(d)


def _small_problem(n=16, V=24, nb=23, M=4, P_=1, seed=11, counts=2e4, pixel_mm=4.0):
    from paper_2111_07886_gb300 import synth
    w = synth.Workload("t", n, P_, pixel_mm, V, nb, pixel_mm, M, counts, "ellipses2d",
                       synth.AlgoParams(), seed=seed)
    scan = synth.make_scan(w)
    g = oracle.geom(n, P_, V, nb, M, pixel_mm=pixel_mm, bin_mm=pixel_mm, sens=scan["sens"])
    return g, scan


def test_em_special_case_preserves_counts():
    """M = 1, beta = 0, gamma -> 0, lambda = alpha = nu = 1, U large: the step is
    Shepp-Vardi EM, f <- f A^T(g / A f) / A^T 1, so sum_j (A^T 1)_j f_j = sum_i g_i after
    every iteration."""
    n, V, nb = 16, 20, 25
    g = oracle.geom(n, 1, V, nb, 1, pixel_mm=2.0, sens=3.0)
    rng = np.random.default_rng(2)
    ones_proj = oracle.forward(g, -1, np.ones((1, n, n)))
    hit = ones_proj > 0
    counts = np.where(hit, rng.integers(1, 50, ones_proj.shape), 0).astype(np.int32)
    gamma = np.full(ones_proj.shape, 1e-30, np.float32)
    sens_img = oracle.back(g, -1, np.ones_like(ones_proj))
    prm = P(iterations=1, beta=0.0, t=1e-300, U=1e300, lambda0=1.0, a=0.0, precond=0)
    f = np.ones((1, n, n))
    for it in range(6):
        f, _ = oracle.reconstruct(g, counts, gamma, prm, f)
        assert abs(np.vdot(sens_img, f) - counts.sum()) < 1e-12 * counts.sum()


def test_box_invariant_and_upper_branch():
    """Every iterate stays strictly inside the box B, 0 < f < U (Eq. OperatorPt maps
    f <= 0 to t and f >= U to U - t and keeps everything else); a small U exercises the
    (U - f)/p branch of Eq. preconditioner and the U - t clamp."""
    g, scan = _small_problem()
    for U in (1000.0, 2.5):
        prm = P(iterations=3, U=U)
        f = np.ones((1, g.n, g.n))
        for J in range(12):
            f, _ = oracle.reconstruct(g, scan["counts"], scan["gamma"], prm, np.ones((1, g.n, g.n)), nsub=J + 1)
            assert f.min() > 0.0 and f.max() < U
        if U < 10:
            assert (f > U / 2).any()


def test_bsrem_is_alpha_nu_one():
    """SDP-BSREM with alpha = nu = 1 (KM with rho = delta = 1 and nu1 = nu2 = 1) is BSREM."""
    g, scan = _small_problem()
    f0 = np.ones((1, g.n, g.n))
    a, _ = oracle.reconstruct(g, scan["counts"], scan["gamma"], P(precond=0, iterations=3), f0)
    b, _ = oracle.reconstruct(g, scan["counts"], scan["gamma"],
                              P(precond=4, iterations=3, rho=1.0, delta1=1.0, delta2=1.0,
                                nu1=1.0, nu2=1.0, J0=0), f0)
    np.testing.assert_array_equal(a, b)


def test_objective_decreases():
    """Phi(f^k) decreases (Sec. III, App. B): strictly for M = 1 with a small step, and
    overall for the SDP-P2 setting of Table II."""
    g, scan = _small_problem(M=1)
    _, obj = oracle.reconstruct(g, scan["counts"], scan["gamma"],
                                P(iterations=8, precond=0, lambda0=0.1, a=0.0),
                                np.ones((1, g.n, g.n)), with_objective=True)
    assert np.all(np.diff(obj) < 0), obj
    g, scan = _small_problem(M=4)
    _, obj = oracle.reconstruct(g, scan["counts"], scan["gamma"], P(iterations=10),
                                np.ones((1, g.n, g.n)), with_objective=True)
    assert obj[-1] < obj[0] and np.all(np.diff(obj[5:]) <= 1e-9 * abs(obj[0])), obj


@pytest.mark.parametrize("kind,U", [(0, 1000.0), (0, 0.0), (4, 1000.0), (3, 1000.0)])
def test_converges_to_lbfgsb_minimiser(kind, U):
    """Theorem 2: SDP-BSREM converges to the unique minimiser of Phi on B.  Reference:
    scipy L-BFGS-B on Phi built from the dense clipping matrix (independent of the oracle's
    projector and objective code).  The phantom fills the image so the minimiser is
    interior, and beta is large enough for BSREM to get close in a few hundred iterations;
    the oracle's Phi must also equal the independent Phi.  U = 0 stands for a tight box,
    U = 1.3 max(f*), where the (U - f)/p branch of Eq. preconditioner is active; kinds 3/4
    are SDP-P1/P2 (Nesterov / KM alpha with nu, frozen after J1 = 300)."""
    from scipy.optimize import minimize
    n, V, nb, M = 8, 24, 15, 3
    g = oracle.geom(n, 1, V, nb, M, pixel_mm=4.0, sens=50.0)
    A = dense_A(n, V, nb) * g.sens * g.pixel_mm
    rng = np.random.default_rng(0)
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
        t = 2 * d / den - d * d * (1 + gr * np.sign(d)) / den ** 2     # d/df_J of pair term
        u = -2 * d / den - d * d * (1 - gr * np.sign(d)) / den ** 2    # d/df_K of pair term
        gr_ = np.zeros_like(f)
        np.add.at(gr_, J, t)
        np.add.at(gr_, K, u)
        return val, gd + beta * gr_

    res = minimize(phi, np.ones(n * n), jac=True, method="L-BFGS-B",
                   bounds=[(0, 1000)] * (n * n), options=dict(maxiter=20000, ftol=1e-15, gtol=1e-12))
    fstar = res.x
    assert fstar.min() > 0.1
    o = oracle.objective(g, counts, gamma, fstar.reshape(1, n, n), beta)
    assert abs(o["phi"] - res.fun) < 1e-12 * abs(res.fun)
    if U == 0.0:
        U = 1.3 * fstar.max()
    if kind == 0:
        prm = P(iterations=400, precond=0, a=1 / 35, beta=beta, U=U)
    else:
        prm = P(iterations=400, precond=kind, a=1 / 35, rho=4.0, delta1=3.0, delta2=3.0,
                nu1=0.8, nu2=1.8, beta=beta, U=U, J1=300)
    f, _ = oracle.reconstruct(g, counts, gamma, prm, np.ones((1, n, n)))
    if U < 10:
        assert f.max() > U / 2
    rel = np.linalg.norm(f.ravel() - fstar) / np.linalg.norm(fstar)
    assert rel < 5e-3, rel
