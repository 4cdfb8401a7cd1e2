"""The paper's convergence experiment (Sec. IV-B) on the GPU path.

Reproduces, with this library's CUDA kernels, the comparisons of Sec. IV-B on 2-D data:

* preconditioners P1 / P2 against their momentum-only surrogates M1 / M2 (Fig. 3: objective
  against time, brain phantom, high count, 12 and 24 subsets);
* SDP-P1 / SDP-P2 against BSREM (Figs. 4-5: global NRMSD against iterations and objective
  against time, 12 and 24 subsets, high and low count);
* ROI NRMSD on the uniform phantom (Fig. 6: 4 hot spheres, 2 cold spheres, a background disk
  and all of them, high count, 24 subsets).

Setup of Sec. IV-A: 256 x 256 pixels of 1.17 mm, 288 views over [0, pi), the bins of a ring of
576 detectors of 4 mm (radius 366.7 mm) sampled every half detector (2 mm of arc; 155 bins cover
the 300 mm field of view) with 32 parallel rays across each bin, the same system matrix to
simulate and to reconstruct, phantom blurred in image space by a Gaussian PSF of FWHM 6.59 mm
before projection, scatter as
a heavily smoothed projection scaled to SF = S/(T+S) = 0.25, randoms uniform at
RF = R/(T+S+R) = 0.25, total counts 6.8e6 (high) / 6.8e5 (low), one Poisson realisation; the
expected scatter + randoms form the background gamma of the reconstruction.  Uniform water
attenuation (0.096 / cm) on the phantom's body outline attenuates the trues by
a_i = exp(-mu x chord_i), and the reconstructions use the system matrix diag(a) A (the same
matrix that simulated the data, as in the paper).  The paper's brain
phantom (a clinical image) is not available: a seeded random-ellipse phantom stands in for it.
beta = 0.1 (high) / 0.8 (low), gamma_R = 2, eps = 1e-12, t = 1e-4, f^0 = 1, lambda_0 = 1,
J0 = 3, J1 = 1000, delta_2 = delta_1, and the a, rho, delta_1, nu_1, nu_2 of Table II and of the
M1 / M2 paragraph of Sec. IV-B.  f^inf is BSREM(24) after 1000 iterations.

Times are GPU time of the subiterations (CUDA events around each iteration's M subiterations;
the objective evaluations for the curves are not counted), so "faster" compares the methods'
cost on the same kernels.

Run:  python -m paper_2111_07886_gb300.convergence --out curves.json [--iterations 60]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import time

import numpy as np

from . import pet, synth

FWHM_MM = 6.59
SF = RF = 0.25
N, PIXEL_MM, VIEWS = 256, 1.17, 288
RING_MM = 576 * 4.0 / (2.0 * math.pi)          # 576 detectors of 4 mm
BIN_MM = math.pi * RING_MM / 576               # half a detector of arc: 2 mm
NBINS = 155                      # odd; the outermost bins reach Rd sin(77.5 dbeta) = 150.4 mm
SUBRAYS = 32                     # parallel rays per detector pair


def geometry(M: int, sens: float):
    return pet.Geometry(N, 1, PIXEL_MM, VIEWS, NBINS, BIN_MM, M, sens, subrays=SUBRAYS,
                        ring_mm=RING_MM)

# Table II (brain column) and the M1 / M2 settings of Sec. IV-B ("Comparison of
# Preconditioners"), as (precond, overrides); delta_2 = delta_1 throughout (Sec. IV-A).
def _p(kind, **kw):
    if "delta1" in kw:
        kw["delta2"] = kw["delta1"]
    return dict(precond=kind, **kw)


BRAIN = {
    "high": {
        12: {"BSREM": _p(0, a=1 / 400), "SDP-P1": _p(3, a=1 / 13, nu1=1.6, nu2=2.4),
             "SDP-P2": _p(4, a=1 / 5, rho=5.0, delta1=5.0, nu1=0.8, nu2=2.2),
             "SDP-M1": _p(1, a=1 / 50), "SDP-M2": _p(2, a=1 / 15, rho=3.0, delta1=1.0)},
        24: {"BSREM": _p(0, a=1 / 35), "SDP-P1": _p(3, a=0.35, nu1=1.6, nu2=2.4),
             "SDP-P2": _p(4, a=0.45, rho=4.0, delta1=3.0, nu1=0.8, nu2=1.8),
             "SDP-M1": _p(1, a=1 / 6), "SDP-M2": _p(2, a=1 / 5, rho=2.6, delta1=0.5)},
    },
    "low": {
        12: {"BSREM": _p(0, a=1 / 18), "SDP-P1": _p(3, a=0.5, nu1=1.6, nu2=2.4),
             "SDP-P2": _p(4, a=1.3, rho=7.5, delta1=5.0, nu1=1.3, nu2=2.1)},
        24: {"BSREM": _p(0, a=1 / 5), "SDP-P1": _p(3, a=1.3, nu1=1.4, nu2=2.5),
             "SDP-P2": _p(4, a=1.4, rho=2.2, delta1=1.0, nu1=1.3, nu2=2.4)},
    },
}
UNIFORM = {"BSREM": _p(0, a=1 / 35), "SDP-P1": _p(3, a=0.5, nu1=1.8, nu2=2.5),
           "SDP-P2": _p(4, a=0.7, rho=3.0, delta1=7.0, nu1=1.4, nu2=2.3)}
COUNTS = {"high": 6.8e6, "low": 6.8e5}
BETA = {"high": 0.1, "low": 0.8}


def _gauss1d(x, sigma, axis):
    """Gaussian smoothing along one axis (zero outside), by direct convolution."""
    r = int(math.ceil(4 * sigma))
    k = np.exp(-0.5 * (np.arange(-r, r + 1) / sigma) ** 2)
    k /= k.sum()
    return np.apply_along_axis(lambda v: np.convolve(v, k, mode="same"), axis, x)


MU_WATER_PER_MM = 0.0096


def simulate(phantom_planes, seed: int, total_counts: float, device) -> dict:
    """Data of Sec. IV-A: trues from the PSF-blurred phantom projected by this library's own
    system model (the paper simulates and reconstructs with the same matrix) and attenuated by
    water on the body outline, scatter, randoms, Poisson noise.  Returns counts, gamma (expected
    scatter + randoms), the attenuation factors mult, the geometry sens and the unblurred pixel
    phantom."""
    import torch
    f_true = synth.rasterize(phantom_planes, N, PIXEL_MM)[0]
    sigma_px = FWHM_MM / (2.0 * math.sqrt(2.0 * math.log(2.0))) / PIXEL_MM
    blurred = _gauss1d(_gauss1d(f_true, sigma_px, 0), sigma_px, 1)
    g1 = geometry(1, 1.0)
    d_img = torch.from_numpy(blurred[None].astype(np.float32)).to(device)
    d_proj = torch.empty((1, VIEWS, NBINS), dtype=torch.float32, device=device)
    pet.forward_subset(g1, -1, d_img, d_proj)
    torch.cuda.synchronize()
    g1.close()
    body = [[(cx, cy, a, b, phi, 1.0) for (cx, cy, a, b, phi, _) in pl[:1]] for pl in phantom_planes]
    offs = synth.ring_offsets_mm(NBINS, BIN_MM, RING_MM)
    mult = np.exp(-MU_WATER_PER_MM * synth.analytic_sinogram(body, VIEWS, NBINS, BIN_MM, offs)[0])
    trues = mult * d_proj.cpu().double().numpy()[0]
    # scatter: the projection smoothed heavily along the bins (FWHM 1/4 of the field), scaled to
    # S = T SF / (1 - SF); randoms uniform, R = (T + S) RF / (1 - RF); all scaled to TC
    scat = _gauss1d(trues, NBINS / 4.0 / 2.355, 1)
    T = trues.sum()
    scat *= T * SF / (1 - SF) / scat.sum()
    R = (T + scat.sum()) * RF / (1 - RF)
    rnd = np.full_like(trues, R / trues.size)
    s = total_counts / (T + scat.sum() + R)
    lam = s * (trues + scat + rnd)
    gamma = (s * (scat + rnd)).astype(np.float32)
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = rng.poisson(lam).astype(np.int32)
    return dict(counts=counts[None], gamma=gamma[None], mult=mult[None].astype(np.float32),
                sens=float(s), f_true=f_true)


def params(base: dict, beta: float, iterations: int):
    p = synth.AlgoParams(iterations=iterations, beta=beta, J0=3, J1=1000)
    return dataclasses.replace(p, **base)


def run(g, d_counts, d_gamma, prm, iterations, device, f_inf=None, rois=None, d_mult=None):
    """One reconstruction, subiteration by subiteration: per iteration the GPU time of its M
    subiterations (CUDA events), Phi(f^k), and NRMSD against f_inf (global and per ROI)."""
    import torch
    f0 = torch.ones((1, N, N), dtype=torch.float32, device=device)
    st = pet.State(g, d_counts, d_gamma, pet.make_params(prm), f0, d_mult=d_mult)
    img = torch.empty_like(f0)
    M = g.nsubsets
    out = {"phi": [st.objective()[0]], "gpu_s": [0.0], "nrmsd": [], "roi_nrmsd": {}}
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t = 0.0
    for k in range(iterations):
        a.record()
        for _ in range(M):
            st.subiter()
        b.record()
        torch.cuda.synchronize()
        t += a.elapsed_time(b) / 1e3
        out["gpu_s"].append(t)
        out["phi"].append(st.objective()[0])
        if f_inf is not None:
            st.read_image(img)
            f = img.cpu().double().numpy()[0]
            out["nrmsd"].append(float(np.linalg.norm(f - f_inf) / np.linalg.norm(f_inf)))
            for name, m in (rois or {}).items():
                out["roi_nrmsd"].setdefault(name, []).append(
                    float(np.linalg.norm(f[m] - f_inf[m]) / np.linalg.norm(f_inf[m])))
    if f_inf is None:
        st.read_image(img)
        out["image"] = img.cpu().double().numpy()[0]
    st.close()
    return out


def reach(phi, target):
    """First iteration k with Phi(f^k) <= target (None if never)."""
    for k, v in enumerate(phi):
        if v <= target:
            return k
    return None


def speedups(curves: dict, ref: str, iters: int) -> dict:
    """Iterations and GPU time each method needs to reach the objective `ref` reaches at its
    last iteration, and the ratio ref / method (the paper's 'faster by a factor')."""
    target = curves[ref]["phi"][iters]
    out = {"target_phi": target, "ref": ref}
    for name, c in curves.items():
        k = reach(c["phi"], target)
        out[name] = {"iterations": k, "gpu_s": c["gpu_s"][k] if k is not None else None,
                     "iteration_ratio": (iters / k) if k else None,
                     "time_ratio": (curves[ref]["gpu_s"][iters] / c["gpu_s"][k]) if k else None}
    return out


def experiment(iterations: int = 60, ref_iterations: int = 1000, seed: int = 0, device=None) -> dict:
    import torch
    device = device or torch.device("cuda")
    res = {"setup": {"image": [N, N], "pixel_mm": PIXEL_MM, "views": VIEWS, "bins": NBINS,
                     "ring": f"radius {RING_MM:.1f} mm, {BIN_MM:.2f} mm of arc per bin, {SUBRAYS} rays per bin",
                     "psf_fwhm_mm": FWHM_MM, "SF": SF, "RF": RF, "iterations": iterations,
                     "attenuation": f"water, {MU_WATER_PER_MM} / mm on the body outline",
                     "f_inf": f"BSREM(24), {ref_iterations} iterations", "seed": seed,
                     "time": "GPU time of the subiterations (CUDA events)"},
           "brain_standin": {}, "uniform": {}}
    t_wall = time.time()
    for level in ("high", "low"):
        data = simulate(synth.brain_standin_2d(N, PIXEL_MM, seed), seed + 11, COUNTS[level], device)
        d_c = torch.from_numpy(data["counts"]).to(device)
        d_g = torch.from_numpy(data["gamma"]).to(device)
        d_m = torch.from_numpy(data["mult"]).to(device)
        beta = BETA[level]
        g24 = geometry(24, data["sens"])
        f_inf = run(g24, d_c, d_g, params(BRAIN[level][24]["BSREM"], beta, ref_iterations),
                    ref_iterations, device, d_mult=d_m)["image"]
        for M in (12, 24):
            g = g24 if M == 24 else geometry(M, data["sens"])
            curves = {}
            for name, base in BRAIN[level][M].items():
                curves[name] = run(g, d_c, d_g, params(base, beta, iterations), iterations, device,
                                   f_inf=f_inf, d_mult=d_m)
            key = f"{level}_{M}"
            res["brain_standin"][key] = {"curves": curves,
                                         "vs_bsrem": speedups(curves, "BSREM", iterations)}
            if "SDP-M1" in curves:
                pm = {}
                for p_, m_ in (("SDP-P1", "SDP-M1"), ("SDP-P2", "SDP-M2")):
                    sp = speedups({p_: curves[p_], m_: curves[m_]}, m_, iterations)
                    pm[f"{p_}_vs_{m_}"] = sp[p_]
                res["brain_standin"][key]["p_vs_m"] = pm
    # uniform phantom, high count, 24 subsets (Fig. 6)
    data = simulate(synth.uniform_phantom_2d(N, PIXEL_MM), seed + 23, COUNTS["high"], device)
    d_c = torch.from_numpy(data["counts"]).to(device)
    d_g = torch.from_numpy(data["gamma"]).to(device)
    d_m = torch.from_numpy(data["mult"]).to(device)
    g24 = geometry(24, data["sens"])
    f_inf = run(g24, d_c, d_g, params(UNIFORM["BSREM"], BETA["high"], ref_iterations),
                ref_iterations, device, d_mult=d_m)["image"]
    rois = synth.uniform_phantom_rois(N, PIXEL_MM)
    curves = {name: run(g24, d_c, d_g, params(base, BETA["high"], iterations), iterations, device,
                        f_inf=f_inf, rois=rois, d_mult=d_m) for name, base in UNIFORM.items()}
    res["uniform"]["high_24"] = {"curves": curves, "vs_bsrem": speedups(curves, "BSREM", iterations)}
    res["setup"]["wall_s"] = round(time.time() - t_wall, 1)
    return res


def summary(res: dict) -> list[str]:
    """One line per comparison: how many times fewer iterations (and less GPU time) a method
    needs to reach the objective the reference reaches at the last iteration."""
    lines = []
    for ph in ("brain_standin", "uniform"):
        for key, r in res[ph].items():
            sp = r["vs_bsrem"]
            for name in ("SDP-P1", "SDP-P2"):
                s = sp[name]
                lines.append(f"{ph} {key} {name} vs BSREM: reaches BSREM's Phi at iteration "
                             f"{s['iterations']} (ratio {s['iteration_ratio']}, time ratio {s['time_ratio']})")
            for k, s in r.get("p_vs_m", {}).items():
                lines.append(f"{ph} {key} {k}: iteration {s['iterations']} "
                             f"(ratio {s['iteration_ratio']}, time ratio {s['time_ratio']})")
    return lines


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", default="convergence_curves.json")
    ap.add_argument("--iterations", type=int, default=60)
    ap.add_argument("--ref-iterations", type=int, default=1000)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    res = experiment(a.iterations, a.ref_iterations, a.seed)
    with open(a.out, "w") as fh:
        json.dump(res, fh)
    for line in summary(res):
        print(line)


if __name__ == "__main__":
    main()
