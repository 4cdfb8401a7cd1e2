"""The paper's simulated data model (Sec. IV-A) in the seeded generator (no GPU): scatter and
random fractions, water attenuation factors of the body's chord, and the PSF width."""
import math

import numpy as np

from paper_2111_07886_gb300 import synth


def _w(**kw):
    d = dict(name="p", n=96, nplanes=1, pixel_mm=3.0, nviews=60, nbins=141, bin_mm=3.0,
             nsubsets=6, counts=6.8e5, phantom="ellipses2d", params=synth.AlgoParams(), seed=4)
    d.update(kw)
    return synth.Workload(**d)


def test_fractions_and_total():
    d = synth.make_scan_paper(_w())
    T, S, R = d["trues"].sum(), d["scatter"].sum(), d["randoms"].sum()
    assert abs(S / (T + S) - 0.25) < 1e-12
    assert abs(R / (T + S + R) - 0.25) < 1e-12
    assert abs(T + S + R - 6.8e5) < 1e-6 * 6.8e5
    np.testing.assert_allclose(d["gamma"], (d["scatter"] + d["randoms"]).astype(np.float32))
    assert np.ptp(d["randoms"]) == 0.0
    # Poisson counts around the mean
    assert abs(d["counts"].sum() - 6.8e5) < 5 * math.sqrt(6.8e5)


def test_attenuation_of_the_centred_water_disk():
    """The 2-D phantom's body is a centred disk of radius 0.45 FOV: a_i = exp(-mu 2 sqrt(R^2 - r^2))
    inside it and 1 outside."""
    w = _w()
    d = synth.make_scan_paper(w)
    rb = 0.45 * w.n * w.pixel_mm
    r = (np.arange(w.nbins) - (w.nbins - 1) / 2.0) * w.bin_mm
    want = np.exp(-synth.PAPER_MU_WATER_PER_MM * 2.0 * np.sqrt(np.clip(rb * rb - r * r, 0, None)))
    np.testing.assert_allclose(d["mult"][0], np.broadcast_to(want, (w.nviews, w.nbins)), rtol=1e-6)
    assert d["mult"].max() == 1.0 and d["mult"].min() > 0.0


def test_psf_blur_width():
    """The 1-D blur that stands for the image-space PSF has the stated FWHM."""
    step = 0.05
    prof = np.zeros(4001)
    prof[2000] = 1.0
    out = synth._gauss_blur_r(prof, step, synth.PAPER_PSF_FWHM_MM)
    assert abs(out.sum() - 1.0) < 1e-12
    above = np.nonzero(out >= 0.5 * out.max())[0]
    fwhm = (above[-1] - above[0] + 1) * step
    assert abs(fwhm - synth.PAPER_PSF_FWHM_MM) <= 2 * step


def test_tof_line_integrals_add_up_to_the_plain_ones():
    """TOF bins covering the image split each exact line integral: their sum is the chord
    integral, and a centred disk puts its TOF profile symmetric about the line's centre."""
    pl = synth.ellipse_phantom_2d(64, 4.0, 3)
    a = synth.analytic_sinogram(pl, 30, 91, 4.0)
    b = synth.analytic_tof_sinogram(pl, 30, 91, 4.0, 41, 12.0, 40.0)
    assert np.abs(b.sum(-1) - a).max() <= 1e-12 * a.max()
    disk = [[(0.0, 0.0, 50.0, 50.0, 0.0, 1.0)]]
    d = synth.analytic_tof_sinogram(disk, 8, 31, 4.0, 21, 10.0, 30.0)
    np.testing.assert_allclose(d, d[..., ::-1], rtol=0, atol=1e-12 * d.max())
