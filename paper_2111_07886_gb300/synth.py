"""Seeded synthetic PET workloads (phantoms, sinograms, algorithm parameters).

This module is the ONLY code shared by the CUDA path and the FP64 oracle, and it holds
none of the reconstruction method's arithmetic: it draws phantoms from a seeded
``numpy.random.Generator(PCG64(seed))``, computes their *analytic* line integrals
(continuous ellipses and ellipsoid cross-sections, not the pixel system matrix), and
draws Poisson counts.  It follows the data model g = Poisson(A f + gamma) of Sec. II-A
(Eq. model-Poisson) with a uniform background gamma > 0.

Geometry conventions (shared by both sides as *definitions*, not code):
  * image N x N pixels of side ``pixel_mm``, centred at the origin; pixel (ix, iy)
    covers [ix - N/2, ix + 1 - N/2) x [iy - N/2, iy + 1 - N/2) in pixel units; the
    flat index is iy * N + ix (x fastest); planes are stacked 2-D slices;
  * view v has angle theta_v = v * pi / V over [0, pi); bin b sits at offset
    r_b = (b - (n_b - 1) / 2) * bin_mm from the centre; ray (v, b) is the line
    {X cos(theta) + Y sin(theta) = r_b};
  * subset i (0-based) holds the views v with v mod M == i (interleaved);
  * the system matrix is A_ij = sens * (length in mm of ray i inside pixel j), so
    ``sens`` converts activity x mm into expected counts.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload", "AlgoParams", "config_2d_128", "config_stacked_256x89",
    "mixed_2d_scans", "make_scan", "ellipse_phantom_2d", "ellipsoid_phantom_3d",
    "rasterize", "random_image", "uniform_phantom_2d", "uniform_phantom_rois",
    "brain_standin_2d", "make_scan_paper", "analytic_tof_sinogram", "ring_offsets_mm",
]

# Preconditioner kinds (Sec. III: BSREM, momentum-only M1/M2, SDP P1/P2).
PRECOND_BSREM, PRECOND_M1, PRECOND_M2, PRECOND_P1, PRECOND_P2 = 0, 1, 2, 3, 4
# Arithmetic of the GPU path.
PREC_FP32, PREC_FP32_KAHAN, PREC_FP64 = 0, 1, 2


@dataclasses.dataclass
class AlgoParams:
    """Parameters of SDP-BSREM (Table I, Eqs. preconditioner:Nesterov/KM, nuki, Table II)."""
    iterations: int = 10
    beta: float = 0.05
    gamma_r: float = 2.0          # Sec. IV-A: gamma_R = 2
    eps: float = 1e-12            # Sec. IV-A: epsilon = 1e-12
    t: float = 1e-4               # Sec. IV-A: t = 1e-4 in P_t
    U: float = 1000.0             # bound of the box B (Eq. BoundedSet); no value in the paper
    lambda0: float = 1.0          # Sec. IV-A: lambda_0 = 1
    a: float = 0.45               # relaxation lambda_k = lambda_0 / (a k + 1)
    rho: float = 2.0              # KM alpha limit (Eq. preconditioner:KM)
    delta1: float = 5.0
    delta2: float = 5.0           # Sec. IV-A: delta_1 = delta_2
    nu1: float = 0.8
    nu2: float = 1.5
    J0: int = 3                   # Sec. IV-A
    J1: int = 1000                # Sec. IV-A prints "J_2 = 1000"; Eq. nuki uses J_1
    precond: int = PRECOND_P2
    precision: int = PREC_FP32_KAHAN
    rdp3d: int = 0                # 0: 8 in-plane neighbours (Sec. IV-A); 1: 26 neighbours in 3-D
    reg: int = 0                  # 0: RDP by its gradient (the paper); 1: TV by a proximal step
    tv_iters: int = 10            # primal-dual iterations per proximal step (reg = 1)


@dataclasses.dataclass
class Workload:
    name: str
    n: int
    nplanes: int
    pixel_mm: float
    nviews: int
    nbins: int
    bin_mm: float
    nsubsets: int
    counts: float                 # expected total counts (signal + background)
    phantom: str                  # "ellipses2d" | "ellipsoid3d"
    params: AlgoParams
    plane_mm: float = 0.0
    seed: int = 0
    subrays: int = 1              # parallel lines per bin of the system model (Sec. IV-A: 32)
    tof_bins: int = 0             # time-of-flight bins per bin (0: no TOF)
    tof_bin_mm: float = 0.0       # TOF bin width along the line
    tof_fwhm_mm: float = 0.0      # FWHM of the timing kernel along the line

    def geometry(self) -> dict:
        return dict(n=self.n, nplanes=self.nplanes, pixel_mm=self.pixel_mm,
                    nviews=self.nviews, nbins=self.nbins, bin_mm=self.bin_mm,
                    nsubsets=self.nsubsets, subrays=self.subrays, tof_bins=self.tof_bins,
                    tof_bin_mm=self.tof_bin_mm, tof_fwhm_mm=self.tof_fwhm_mm)


# SDP-P2 settings of the workloads.  Table II's rows were tuned on the paper's brain phantom;
# on these synthetic scans its high-count P2 rows (rho = 5 / 4) drive lambda alpha nu far above
# one in the first iteration, f~ dips below zero all over the background, and the jump of P_t
# at zero makes the FP64 trajectory itself chaotic (a 1e-10 relative change of f^0 changes
# f^T by O(1)).  The workloads therefore use the P2 form with rho = 2, delta1 = delta2 = 5,
# a = 0.45, nu in [0.8, 1.5]: well conditioned (a 1e-7 change of f^0 moves f^T by < 3e-7)
# with a monotone objective.  Table II's own rows stay available as TABLE2.
P2_WORKLOAD = dict(a=0.45, rho=2.0, delta1=5.0, delta2=5.0, nu1=0.8, nu2=1.5)

TABLE2 = {   # Table II (2-D simulations), high / low count
    "BSREM(12)": (dict(precond=PRECOND_BSREM, a=1 / 400), dict(precond=PRECOND_BSREM, a=1 / 18)),
    "SDP-P1(12)": (dict(precond=PRECOND_P1, a=1 / 13, nu1=1.6, nu2=2.4),
                   dict(precond=PRECOND_P1, a=0.5, nu1=1.6, nu2=2.4)),
    "SDP-P2(12)": (dict(precond=PRECOND_P2, a=1 / 5, rho=5.0, delta1=5.0, delta2=5.0, nu1=0.8, nu2=2.2),
                   dict(precond=PRECOND_P2, a=1.3, rho=7.5, delta1=5.0, delta2=5.0, nu1=1.3, nu2=2.1)),
    "BSREM(24)": (dict(precond=PRECOND_BSREM, a=1 / 35), dict(precond=PRECOND_BSREM, a=1 / 5)),
    "SDP-P1(24)": (dict(precond=PRECOND_P1, a=0.35, nu1=1.6, nu2=2.4),
                   dict(precond=PRECOND_P1, a=1.3, nu1=1.4, nu2=2.5)),
    "SDP-P2(24)": (dict(precond=PRECOND_P2, a=0.45, rho=4.0, delta1=3.0, delta2=3.0, nu1=0.8, nu2=1.8),
                   dict(precond=PRECOND_P2, a=1.4, rho=2.2, delta1=1.0, delta2=1.0, nu1=1.3, nu2=2.4)),
}


def config_2d_128(seed: int = 0) -> Workload:
    """2-D plain method: 128^2 at 4 mm, 180 views x 185 bins, 12 subsets, 1e6 counts,
    10 iterations, RDP weight 0.05, SDP-P2 (P2_WORKLOAD settings)."""
    p = AlgoParams(iterations=10, beta=0.05, **P2_WORKLOAD)
    return Workload("2d_128x128_v180_b185_m12", 128, 1, 4.0, 180, 185, 4.0, 12, 1e6,
                    "ellipses2d", p, seed=seed)


def config_stacked_256x89(seed: int = 0, nplanes: int = 89, iterations: int = 20) -> Workload:
    """Clinical-size stacked 2-D: 256^2 x 89 at 2.7 mm, 288 views x 357 bins, 24 subsets,
    5e7 counts per volume, 20 iterations, RDP weight 0.02, SDP-P2 (P2_WORKLOAD settings)."""
    p = AlgoParams(iterations=iterations, beta=0.02, **P2_WORKLOAD)
    return Workload(f"stacked_256x256x{nplanes}_v288_b357_m24", 256, nplanes, 2.7, 288,
                    357, 2.7, 24, 5e7 * nplanes / 89.0, "ellipsoid3d", p, plane_mm=2.7,
                    seed=seed)


def mixed_2d_scans(count: int = 64, seed: int = 0, iterations: int = 10) -> list[Workload]:
    """Mixed 2-D scans: N in {128, 200, 256, 400} at FOV 512 mm, 120-360 views,
    n_b = largest odd <= 1.45 N (bin = pixel), counts log-uniform in [1e5, 1e7],
    12-36 subsets."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for s in range(count):
        n = int(rng.choice([128, 200, 256, 400]))
        v = int(rng.integers(120, 361))
        nb = int(math.floor(1.45 * n))
        if nb % 2 == 0:
            nb -= 1
        m = int(rng.choice([12, 18, 24, 36]))
        counts = float(10 ** rng.uniform(5, 7))
        p = AlgoParams(iterations=iterations, beta=0.05, **P2_WORKLOAD)
        out.append(Workload(f"mix{s}_{n}_v{v}_b{nb}_m{m}", n, 1, 512.0 / n, v, nb,
                            512.0 / n, m, counts, "ellipses2d", p,
                            seed=seed * 1000 + s + 1))
    return out


# ----------------------------------------------------------------------------------
# Phantoms: lists of ellipses per plane, (cx, cy, ax, ay, phi, value) in mm, additive.
# ----------------------------------------------------------------------------------

def _overlap(c1, r1, c2, r2) -> bool:
    return math.hypot(c1[0] - c2[0], c1[1] - c2[1]) < r1 + r2 + 1e-9


def ellipse_phantom_2d(n: int, pixel_mm: float, seed: int, n_ellipses: int = 10):
    """Disk background of value 1 (radius 0.45 FOV) holding ``n_ellipses`` random,
    non-overlapping ellipses of intensity U[0.5, 4] (the ellipse replaces the background,
    so it is stored as an additive offset intensity - 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fov = n * pixel_mm
    rbg = 0.45 * fov
    shapes = [(0.0, 0.0, rbg, rbg, 0.0, 1.0)]
    placed = []
    tries = 0
    while len(placed) < n_ellipses and tries < 20000:
        tries += 1
        ax, ay = rng.uniform(0.04, 0.2, size=2) * rbg
        rad = 0.7 * rbg * math.sqrt(rng.uniform())
        ang = rng.uniform(0, 2 * math.pi)
        c = (rad * math.cos(ang), rad * math.sin(ang))
        r = max(ax, ay)
        if math.hypot(*c) + r > 0.95 * rbg:
            continue
        if any(_overlap(c, r, c2, r2) for c2, r2 in placed):
            continue
        phi = rng.uniform(0, math.pi)
        val = rng.uniform(0.5, 4.0)
        placed.append((c, r))
        shapes.append((c[0], c[1], ax, ay, phi, val - 1.0))
    return [shapes]


def ellipsoid_phantom_3d(n: int, nplanes: int, pixel_mm: float, plane_mm: float, seed: int,
                         n_spheres: int = 6):
    """Random ellipsoid body (value 1) holding ``n_spheres`` hot spheres of diameter
    U[3, 15] mm at contrast 4:1; returns the elliptical cross-section of every plane."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fov = n * pixel_mm
    ax, ay = rng.uniform(0.28, 0.38) * fov, rng.uniform(0.2, 0.28) * fov
    az = rng.uniform(0.5, 0.7) * max(nplanes * plane_mm, 1.0)
    phi = rng.uniform(0, math.pi)
    spheres = []
    tries = 0
    zext = max(0.5 * (nplanes - 1) * plane_mm, 1.0)
    while len(spheres) < n_spheres and tries < 20000:
        tries += 1
        rad = 0.5 * rng.uniform(3.0, 15.0)
        c = (rng.uniform(-0.6, 0.6) * ax, rng.uniform(-0.6, 0.6) * ay,
             rng.uniform(-0.8, 0.8) * zext)
        if any(math.dist(c, c2) < rad + r2 + 2.0 for c2, r2 in spheres):
            continue
        spheres.append((c, rad))
    planes = []
    for p in range(nplanes):
        z = (p - (nplanes - 1) / 2.0) * plane_mm
        sh = []
        k2 = 1.0 - (z / az) ** 2
        if k2 > 0:
            k = math.sqrt(k2)
            sh.append((0.0, 0.0, ax * k, ay * k, phi, 1.0))
        for (cx, cy, cz), rad in spheres:
            d2 = rad * rad - (z - cz) ** 2
            if d2 > 0:
                rr = math.sqrt(d2)
                sh.append((cx, cy, rr, rr, 0.0, 3.0))
        planes.append(sh)
    return planes


def uniform_phantom_2d(n: int = 256, pixel_mm: float = 1.17):
    """The uniform phantom of Sec. IV-A: a uniform disk background (value 1) holding 4 hot
    spheres (value 10, contrast 1:10) and 2 cold spheres (value 0) of radii 4, 6, 8 (cold),
    10 (cold), 12 and 14 pixels.  The paper gives no positions: the six sphere centres sit on a
    circle of radius 0.25 n pixels, 60 degrees apart, and the background disk has radius
    0.43 n pixels, leaving the centre free for the background ROI."""
    rb = 0.43 * n * pixel_mm
    shapes = [(0.0, 0.0, rb, rb, 0.0, 1.0)]
    for (cx, cy, r, val) in _uniform_spheres(n, pixel_mm):
        shapes.append((cx, cy, r, r, 0.0, val - 1.0))
    return [shapes]


def _uniform_spheres(n: int, pixel_mm: float):
    radii = [(4, 10.0), (6, 10.0), (8, 0.0), (10, 0.0), (12, 10.0), (14, 10.0)]
    out = []
    for k, (r_px, val) in enumerate(radii):
        ang = k * math.pi / 3.0
        c = 0.25 * n * pixel_mm
        out.append((c * math.cos(ang), c * math.sin(ang), r_px * pixel_mm, val))
    return out


def uniform_phantom_rois(n: int = 256, pixel_mm: float = 1.17):
    """The 8 ROIs of the uniform phantom (Fig. 6 of Sec. IV-B): the 4 hot and 2 cold spheres,
    one background disk of radius 25 pixels at the centre, and all 7 together.  Returns
    {name: boolean mask [N][N]} over pixel centres."""
    g = (np.arange(n) + 0.5 - n / 2.0) * pixel_mm
    X, Y = np.meshgrid(g, g)
    rois = {}
    for (cx, cy, r, val) in _uniform_spheres(n, pixel_mm):
        name = f"{'hot' if val > 1 else 'cold'}_r{int(round(r / pixel_mm))}"
        rois[name] = (X - cx) ** 2 + (Y - cy) ** 2 <= r * r
    rois["background_r25"] = X ** 2 + Y ** 2 <= (25 * pixel_mm) ** 2
    allm = np.zeros((n, n), bool)
    for m in rois.values():
        allm |= m
    rois["all"] = allm
    return rois


def brain_standin_2d(n: int = 256, pixel_mm: float = 1.17, seed: int = 0):
    """Stand-in for the paper's brain phantom (a clinical image, not available): the random
    ellipse phantom (disk background 1, ten ellipses of intensity U[0.5, 4])."""
    return ellipse_phantom_2d(n, pixel_mm, seed)


def analytic_sinogram(planes, nviews: int, nbins: int, bin_mm: float, offsets_mm=None) -> np.ndarray:
    """Exact line integrals (activity x mm) of the continuous phantom along every ray,
    [P][V][n_b] float64.  For an ellipse with semi-axes (a, b), rotation phi, centre c,
    the chord along {X cos t + Y sin t = r} is 2ab sqrt(D^2 - r'^2) / D^2 with
    D^2 = a^2 cos^2(t - phi) + b^2 sin^2(t - phi) and r' = r - <c, (cos t, sin t)>.  The
    lines sit at r = (b - (n_b - 1)/2) bin_mm, or at ``offsets_mm`` (n_b values) when given."""
    theta = np.arange(nviews) * math.pi / nviews
    ct, st = np.cos(theta)[:, None], np.sin(theta)[:, None]
    if offsets_mm is None:
        r = ((np.arange(nbins) - (nbins - 1) / 2.0) * bin_mm)[None, :]
    else:
        r = np.asarray(offsets_mm, np.float64)[None, :]
    out = np.zeros((len(planes), nviews, nbins))
    for p, shapes in enumerate(planes):
        for (cx, cy, a, b, phi, val) in shapes:
            d2 = (a * np.cos(theta - phi)) ** 2 + (b * np.sin(theta - phi)) ** 2
            d2 = d2[:, None]
            rp = r - (cx * ct + cy * st)
            inside = np.clip(d2 - rp * rp, 0.0, None)
            out[p] += val * 2.0 * a * b * np.sqrt(inside) / d2
    return out


def ring_offsets_mm(nbins: int, bin_mm: float, ring_mm: float) -> np.ndarray:
    """Line offsets of a view's bins on a detector ring of radius ``ring_mm`` sampled every
    ``bin_mm`` of arc: r_b = ring_mm sin((b - (n_b - 1)/2) bin_mm / ring_mm)."""
    return ring_mm * np.sin((np.arange(nbins) - (nbins - 1) / 2.0) * bin_mm / ring_mm)


def analytic_tof_sinogram(planes, nviews: int, nbins: int, bin_mm: float, tof_bins: int,
                          tof_bin_mm: float, tof_fwhm_mm: float) -> np.ndarray:
    """Exact TOF line integrals [P][V][n_b][T] of the continuous phantom: for every ellipse and
    line, the chord [tau1, tau2] along the line (tau measured from the line's point nearest the
    centre along (-sin t, cos t)) weighted by the TOF bin's kernel h_t(tau) (a Gaussian of FWHM
    ``tof_fwhm_mm`` integrated over the bin), integrated in closed form:
    int Phi((e - tau) / s) dtau = -s Psi((e - tau) / s), Psi(x) = x Phi(x) + phi(x)."""
    from scipy.special import ndtr
    theta = np.arange(nviews) * math.pi / nviews
    ct, st = np.cos(theta)[:, None], np.sin(theta)[:, None]
    r = ((np.arange(nbins) - (nbins - 1) / 2.0) * bin_mm)[None, :]
    sig = tof_fwhm_mm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    edges = (np.arange(tof_bins + 1) - tof_bins / 2.0) * tof_bin_mm

    def psi(x):
        return x * ndtr(x) + np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)

    out = np.zeros((len(planes), nviews, nbins, tof_bins))
    for p, shapes in enumerate(planes):
        for (cx, cy, a, b, phi, val) in shapes:
            ux, uy, wx, wy = math.cos(phi), math.sin(phi), -math.sin(phi), math.cos(phi)
            p0x, p0y = r * ct - cx, r * st - cy                 # line point at tau = 0, from C
            dx, dy = -st, ct                                    # line direction
            du, dw = dx * ux + dy * uy, dx * wx + dy * wy
            pu, pw = p0x * ux + p0y * uy, p0x * wx + p0y * wy
            A = du * du / a ** 2 + dw * dw / b ** 2
            B = 2.0 * (pu * du / a ** 2 + pw * dw / b ** 2)
            C = pu * pu / a ** 2 + pw * pw / b ** 2 - 1.0
            disc = B * B - 4.0 * A * C
            hit = disc > 0
            sq = np.sqrt(np.where(hit, disc, 0.0))
            t1 = np.where(hit, (-B - sq) / (2.0 * A), 0.0)
            t2 = np.where(hit, (-B + sq) / (2.0 * A), 0.0)
            # int_{t1}^{t2} Phi((e - tau) / sig) dtau at every edge e
            F = np.stack([sig * (psi((e - t1) / sig) - psi((e - t2) / sig)) for e in edges], -1)
            out[p] += val * (F[..., 1:] - F[..., :-1])
    return out


def rasterize(planes, n: int, pixel_mm: float, supersample: int = 4) -> np.ndarray:
    """Pixel image [P][N][N] of the phantom (partial volume by supersampling)."""
    s = supersample
    g = (np.arange(n * s) + 0.5) / s - n / 2.0
    X, Y = np.meshgrid(g * pixel_mm, g * pixel_mm)
    out = np.zeros((len(planes), n, n))
    for p, shapes in enumerate(planes):
        img = np.zeros_like(X)
        for (cx, cy, a, b, phi, val) in shapes:
            dx, dy = X - cx, Y - cy
            u = dx * math.cos(phi) + dy * math.sin(phi)
            w = -dx * math.sin(phi) + dy * math.cos(phi)
            img += val * ((u / a) ** 2 + (w / b) ** 2 <= 1.0)
        out[p] = img.reshape(n, s, n, s).mean(axis=(1, 3))
    return out


def make_scan(w: Workload) -> dict:
    """Counts (int32 [P][V][n_b]), background gamma (float32, uniform, 10 % of the mean
    signal), the projector scale ``sens`` and the phantom, for workload ``w``.

    ``sens`` is chosen so that the expected total counts sum(sens * line integrals)
    + sum(gamma) equals ``w.counts``."""
    if w.phantom == "ellipses2d":
        planes = ellipse_phantom_2d(w.n, w.pixel_mm, w.seed)
    else:
        planes = ellipsoid_phantom_3d(w.n, w.nplanes, w.pixel_mm, w.plane_mm, w.seed)
    if w.tof_bins > 1:
        sino = analytic_tof_sinogram(planes, w.nviews, w.nbins, w.bin_mm, w.tof_bins,
                                     w.tof_bin_mm, w.tof_fwhm_mm)
    else:
        sino = analytic_sinogram(planes, w.nviews, w.nbins, w.bin_mm)
    total_signal = sino.sum()
    sens = w.counts / (1.1 * total_signal)
    mean_sig = sens * total_signal / sino.size
    gamma = np.full(sino.shape, 0.1 * mean_sig, dtype=np.float32)
    rng = np.random.Generator(np.random.PCG64(w.seed + 7919))
    lam = sens * sino + gamma.astype(np.float64)
    counts = rng.poisson(lam).astype(np.int32)
    return dict(counts=counts, gamma=gamma, sens=float(sens), planes=planes)


def _gauss_blur_r(prof: np.ndarray, step_mm: float, fwhm_mm: float) -> np.ndarray:
    """Gaussian blur (FWHM ``fwhm_mm``) of profiles sampled every ``step_mm`` along the last
    axis (zero outside), as a normalised discrete convolution."""
    sigma = fwhm_mm / (2.0 * math.sqrt(2.0 * math.log(2.0))) / step_mm
    half = int(math.ceil(5.0 * sigma))
    k = np.exp(-0.5 * (np.arange(-half, half + 1) / sigma) ** 2)
    k /= k.sum()
    flat = prof.reshape(-1, prof.shape[-1])
    out = np.stack([np.convolve(row, k, mode="same") for row in flat])
    return out.reshape(prof.shape)


PAPER_PSF_FWHM_MM = 6.59        # Sec. IV-A: shift-invariant Gaussian PSF of the data
PAPER_MU_WATER_PER_MM = 0.0096  # Sec. IV-A: water attenuation 0.096 / cm
PAPER_SF = PAPER_RF = 0.25      # Sec. IV-A: scatter and random fractions


def make_scan_paper(w: Workload, psf_fwhm_mm: float = PAPER_PSF_FWHM_MM,
                    mu_per_mm: float = PAPER_MU_WATER_PER_MM, sf: float = PAPER_SF,
                    rf: float = PAPER_RF, scatter_fwhm_mm: float = 150.0,
                    oversample: int = 8) -> dict:
    """The data model of the paper's simulations (Sec. IV-A) for workload ``w``:

      * trues: the projection of the phantom convolved with a Gaussian PSF of FWHM
        ``psf_fwhm_mm``; for an isotropic Gaussian the line integrals of the blurred image are the
        analytic line integrals blurred by the same 1-D Gaussian along the detector axis
        (projection-slice theorem), computed on a grid ``oversample`` times finer than the bins
        and sampled at the bin centres; attenuated by a_i = exp(-mu L_i), L_i the chord of the
        phantom's body (its first, outline shape: uniform water on the image's support);
      * scatter: the (unattenuated) projection of the phantom smoothed by a Gaussian of FWHM
        ``scatter_fwhm_mm`` along the detector axis ("highly smoothed"), scaled so that the
        scatter fraction S / (T + S) is ``sf``;
      * randoms: uniform over the sinogram, scaled so that R / (T + S + R) is ``rf``;
      * the total T + S + R is ``w.counts``; counts = Poisson(T + S + R).

    Returns counts (int32), gamma = S + R (float32, the known background), mult = a (float32,
    the per-bin detection factors of the system matrix diag(a) sens L), sens and the phantom.
    The reconstruction model keeps one line per bin (or the workload's sub-rays) and no PSF."""
    if w.phantom == "ellipses2d":
        planes = ellipse_phantom_2d(w.n, w.pixel_mm, w.seed)
    else:
        planes = ellipsoid_phantom_3d(w.n, w.nplanes, w.pixel_mm, w.plane_mm, w.seed)
    fine = w.bin_mm / oversample
    margin = int(math.ceil(3.0 * max(psf_fwhm_mm, scatter_fwhm_mm) / fine))
    nfine = w.nbins * oversample + 2 * margin
    # fine grid centred like the bins: fine sample m sits at (m - (nfine - 1) / 2) * fine
    proj_f = analytic_sinogram(planes, w.nviews, nfine, fine)
    centre = (np.arange(w.nbins) - (w.nbins - 1) / 2.0) * w.bin_mm
    idx = np.rint(centre / fine + (nfine - 1) / 2.0).astype(int)
    trues_shape = _gauss_blur_r(proj_f, fine, psf_fwhm_mm)[..., idx]
    scatter_shape = _gauss_blur_r(proj_f, fine, scatter_fwhm_mm)[..., idx]
    body = [[sh[0]] if sh else [] for sh in planes]
    chord = analytic_sinogram([[(cx, cy, a, b, phi, 1.0) for (cx, cy, a, b, phi, _) in sh]
                               for sh in body], w.nviews, w.nbins, w.bin_mm)
    mult = np.exp(-mu_per_mm * chord)
    t_sino = mult * trues_shape                      # trues per unit sens
    s_scale = sf / (1.0 - sf) * t_sino.sum() / scatter_shape.sum()
    s_sino = s_scale * scatter_shape
    r_total = rf / (1.0 - rf) * (t_sino.sum() + s_sino.sum())
    r_sino = np.full(t_sino.shape, r_total / t_sino.size)
    sens = w.counts / (t_sino.sum() + s_sino.sum() + r_total)
    trues = sens * t_sino
    gamma = (sens * (s_sino + r_sino)).astype(np.float32)
    rng = np.random.Generator(np.random.PCG64(w.seed + 7919))
    counts = rng.poisson(trues + gamma.astype(np.float64)).astype(np.int32)
    return dict(counts=counts, gamma=gamma, mult=mult.astype(np.float32), sens=float(sens),
                planes=planes, trues=trues, scatter=sens * s_sino, randoms=sens * r_sino)


def random_image(shape, seed: int, lo: float = 0.1, hi: float = 2.0) -> np.ndarray:
    """Seeded uniform random image / sinogram (test inputs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=shape)
