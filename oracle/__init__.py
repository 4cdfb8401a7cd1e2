"""FP64 CPU oracle for SDP-BSREM (arXiv 2111.07886) — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It wraps ``pet_oracle.c`` (plain C, double precision, built with gcc)
through ctypes and shares no code with the CUDA library.  See the C file's header for the
passage of the paper each function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pet_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FMA contraction so that x86 and Arm
    round alike)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Geom(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nplanes", ctypes.c_int), ("nviews", ctypes.c_int),
                ("nbins", ctypes.c_int), ("nsubsets", ctypes.c_int),
                ("pixel_mm", ctypes.c_double), ("bin_mm", ctypes.c_double),
                ("sens", ctypes.c_double), ("subrays", ctypes.c_int),
                ("tof_bins", ctypes.c_int), ("tof_bin_mm", ctypes.c_double),
                ("tof_fwhm_mm", ctypes.c_double), ("ring_mm", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int)] + [
        (k, ctypes.c_double) for k in ("beta", "gamma_r", "eps", "t", "U", "lambda0", "a",
                                       "rho", "delta1", "delta2", "nu1", "nu2")] + [
        ("J0", ctypes.c_int), ("J1", ctypes.c_int), ("precond", ctypes.c_int),
        ("rdp3d", ctypes.c_int), ("reg", ctypes.c_int), ("tv_iters", ctypes.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            fp = ctypes.POINTER(ctypes.c_float)
            gp = ctypes.POINTER(Geom)
            L.ora_ray_pieces.argtypes = [gp, ctypes.c_int, ctypes.c_int, ip, dp]
            L.ora_ray_pieces.restype = ctypes.c_int
            L.ora_bin_pieces.argtypes = [gp, ctypes.c_int, ctypes.c_int, ip, dp]
            L.ora_bin_pieces.restype = ctypes.c_int
            L.ora_subset_size.argtypes = [gp, ctypes.c_int]
            L.ora_subset_size.restype = ctypes.c_int
            L.ora_forward.argtypes = [gp, ctypes.c_int, dp, dp]
            L.ora_back.argtypes = [gp, ctypes.c_int, dp, dp]
            L.ora_sensitivity.argtypes = [gp, dp]
            L.ora_rdp_value.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_double]
            L.ora_rdp_value.restype = ctypes.c_double
            L.ora_rdp_grad.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp]
            L.ora_matlab_gradient.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
            L.ora_nu_from_image.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp]
            L.ora_nu_from_image3.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int, dp]
            L.ora_rdp_value3.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_double]
            L.ora_rdp_value3.restype = ctypes.c_double
            L.ora_rdp_grad3.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp]
            L.ora_matlab_gradient_z.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
            L.ora_objective3.argtypes = [gp, ip, fp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, dp]
            L.ora_tv_value.argtypes = [ctypes.c_int, ctypes.c_int, dp]
            L.ora_tv_value.restype = ctypes.c_double
            L.ora_tv_prox.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_int,
                                      dp, dp, dp]
            L.ora_alpha_nesterov.argtypes = [ctypes.c_int, dp]
            L.ora_alpha_km.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            L.ora_objective.argtypes = [gp, ip, fp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            L.ora_reconstruct.argtypes = [gp, ip, fp, ctypes.POINTER(Params), dp, ctypes.c_int, dp]
            L.ora_reconstruct_m.argtypes = [gp, ip, fp, fp, ctypes.POINTER(Params), dp, ctypes.c_int, dp, dp]
            L.ora_objective_m.argtypes = [gp, ip, fp, fp, dp, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, dp]
            L.ora_sensitivity_m.argtypes = [gp, fp, dp]
            L.ora_tof_weight.argtypes = [gp, ctypes.c_int, ctypes.c_double]
            L.ora_tof_weight.restype = ctypes.c_double
            L.ora_reconstruct_snap.argtypes = [gp, ip, fp, ctypes.POINTER(Params), dp, ctypes.c_int, dp, dp]
            _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def geom(n, nplanes, nviews, nbins, nsubsets, pixel_mm=1.0, bin_mm=None, sens=1.0,
         subrays=1, tof_bins=0, tof_bin_mm=0.0, tof_fwhm_mm=0.0, ring_mm=0.0) -> Geom:
    return Geom(n, nplanes, nviews, nbins, nsubsets, pixel_mm,
                pixel_mm if bin_mm is None else bin_mm, sens, subrays, tof_bins, tof_bin_mm,
                tof_fwhm_mm, ring_mm)


def geom_from(geometry: dict, sens: float) -> Geom:
    g = geometry
    return Geom(g["n"], g["nplanes"], g["nviews"], g["nbins"], g["nsubsets"],
                g["pixel_mm"], g["bin_mm"], sens, int(g.get("subrays", 1)),
                int(g.get("tof_bins", 0)), float(g.get("tof_bin_mm", 0.0)),
                float(g.get("tof_fwhm_mm", 0.0)), float(g.get("ring_mm", 0.0)))


def ntof(g: Geom) -> int:
    return g.tof_bins if g.tof_bins > 1 else 1


def tof_weight(g: Geom, t: int, tau_mm: float) -> float:
    """h_t(tau): the Gaussian timing kernel integrated over TOF bin t, at tau mm along a line."""
    return lib().ora_tof_weight(ctypes.byref(g), t, tau_mm)


def subset_size(g: Geom, subset: int) -> int:
    return lib().ora_subset_size(ctypes.byref(g), subset)


def ray_pieces(g: Geom, v: int, b: int):
    """Siddon pieces of ray (v, b): (flat in-plane pixel index, length in pixel units)."""
    cap = 2 * g.n + 2
    pix = np.zeros(cap, np.int32)
    ln = np.zeros(cap, np.float64)
    k = lib().ora_ray_pieces(ctypes.byref(g), v, b,
                             pix.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                             ln.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return pix[:k].copy(), ln[:k].copy()


def bin_pieces(g: Geom, v: int, b: int):
    """Pieces of bin (v, b) under the sub-ray model: every sub-ray's Siddon pieces, lengths / R."""
    cap = max(1, g.subrays) * (2 * g.n + 2)
    pix = np.zeros(cap, np.int32)
    ln = np.zeros(cap, np.float64)
    k = lib().ora_bin_pieces(ctypes.byref(g), v, b,
                             pix.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                             ln.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return pix[:k].copy(), ln[:k].copy()


def forward(g: Geom, subset: int, f) -> np.ndarray:
    """y = A_i f, f [P][N][N] -> [P][V_i][n_b] (subset -1: all views, [P][V][n_b]); with TOF
    bins [P][V_i][n_b][T]."""
    f, fp = _d(f)
    nv = g.nviews if subset < 0 else subset_size(g, subset)
    y = np.zeros((g.nplanes, nv, g.nbins) + ((ntof(g),) if ntof(g) > 1 else ()))
    lib().ora_forward(ctypes.byref(g), subset, fp, y.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return y


def back(g: Geom, subset: int, y) -> np.ndarray:
    """A_i^T y, y [P][V_i][n_b] ([P][V_i][n_b][T] with TOF bins) -> [P][N][N]."""
    y, yp = _d(y)
    out = np.zeros((g.nplanes, g.n, g.n))
    lib().ora_back(ctypes.byref(g), subset, yp, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def sensitivity(g: Geom) -> np.ndarray:
    """p_j of Eq. pj, [N][N]."""
    out = np.zeros((g.n, g.n))
    lib().ora_sensitivity(ctypes.byref(g), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def _fptr(a):
    """float32 [P][V][n_b] per-bin detection factors (or None: all ones) as a C pointer."""
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def sensitivity_m(g: Geom, mult) -> np.ndarray:
    """p_j of Eq. pj for the system matrix diag(mult) A: (A^T mult)_j / M per voxel, [P][N][N]."""
    keep, mp = _fptr(mult)
    out = np.zeros((g.nplanes, g.n, g.n))
    lib().ora_sensitivity_m(ctypes.byref(g), mp, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def rdp_value(f, gamma_r=2.0, eps=1e-12, three_d=False) -> float:
    """R(f) of Eq. RDP: 8 in-plane neighbours, or the 26 neighbours of the volume (three_d)."""
    f, fp = _d(f)
    P, N = (1,) + f.shape if f.ndim == 2 else f.shape[:2]
    fn = lib().ora_rdp_value3 if three_d else lib().ora_rdp_value
    return fn(N, P, fp, gamma_r, eps)


def rdp_grad(f, gamma_r=2.0, eps=1e-12, three_d=False) -> np.ndarray:
    """dR/df of Eq. gradRD over the same neighbourhood as rdp_value."""
    f, fp = _d(f)
    P, N = (1,) + f.shape if f.ndim == 2 else f.shape[:2]
    out = np.zeros_like(f)
    fn = lib().ora_rdp_grad3 if three_d else lib().ora_rdp_grad
    fn(N, P, fp, gamma_r, eps, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def matlab_gradient(f):
    f, fp = _d(f)
    P, N = (1,) + f.shape if f.ndim == 2 else f.shape[:2]
    gx, gy = np.zeros_like(f), np.zeros_like(f)
    lib().ora_matlab_gradient(N, P, fp, gx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              gy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return gx, gy


def matlab_gradient_z(f) -> np.ndarray:
    """Third component of Matlab's gradient of the volume (along the planes)."""
    f, fp = _d(f)
    P, N = f.shape[:2]
    gz = np.zeros_like(f)
    lib().ora_matlab_gradient_z(N, P, fp, gz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return gz


def nu_from_image(f, nu1, nu2, three_d=False) -> np.ndarray:
    f, fp = _d(f)
    P, N = (1,) + f.shape if f.ndim == 2 else f.shape[:2]
    out = np.zeros_like(f)
    lib().ora_nu_from_image3(N, P, fp, nu1, nu2, 1 if three_d else 0,
                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def tv_value(f) -> float:
    """R_TV(f): isotropic total variation, in-plane forward differences (TV variant)."""
    f, fp = _d(f)
    P, N = (1,) + f.shape if f.ndim == 2 else f.shape[:2]
    return lib().ora_tv_value(N, P, fp)


def tv_prox(z, W, b, iters, p=None):
    """Primal-dual approximation of argmin_x 1/2 sum (x - z)^2 / W + b R_TV(x); returns
    (x, (px, py)) with the dual variable updated from `p` (zeros if None)."""
    z, zp = _d(z)
    W, Wp = _d(W)
    P, N = z.shape[:2]
    px = np.zeros_like(z) if p is None else np.array(p[0], dtype=np.float64, order="C")
    py = np.zeros_like(z) if p is None else np.array(p[1], dtype=np.float64, order="C")
    x = np.zeros_like(z)
    dp = ctypes.POINTER(ctypes.c_double)
    lib().ora_tv_prox(N, P, zp, Wp, b, iters, px.ctypes.data_as(dp), py.ctypes.data_as(dp),
                      x.ctypes.data_as(dp))
    return x, (px, py)


def alpha_nesterov(nsub: int) -> np.ndarray:
    out = np.zeros(nsub)
    lib().ora_alpha_nesterov(nsub, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def alpha_km(nsub: int, rho: float, delta1: float, delta2: float) -> np.ndarray:
    out = np.zeros(nsub)
    lib().ora_alpha_km(nsub, rho, delta1, delta2, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def objective(g: Geom, counts, gamma, f, beta, gamma_r=2.0, eps=1e-12, three_d=False,
              tv=False, mult=None) -> dict:
    """Phi(f) and its parts: sum(Af), sum(g ln(Af + gamma)), R(f) (R_TV with tv); with
    ``mult`` the system matrix is diag(mult) A."""
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    gamma = np.ascontiguousarray(gamma, dtype=np.float32)
    keep, mp = _fptr(mult)
    f, fp = _d(f)
    out = np.zeros(4)
    lib().ora_objective_m(ctypes.byref(g), counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          gamma.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), mp, fp, beta,
                          gamma_r, eps, 2 if tv else (1 if three_d else 0),
                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return dict(sum_af=out[0], sum_glog=out[1], rdp=out[2], phi=out[3])


def params_from(p) -> Params:
    """Oracle parameters from an object with the AlgoParams attribute names."""
    return Params(p.iterations, p.beta, p.gamma_r, p.eps, p.t, p.U, p.lambda0, p.a, p.rho,
                  p.delta1, p.delta2, p.nu1, p.nu2, p.J0, p.J1, p.precond,
                  int(getattr(p, "rdp3d", 0)), int(getattr(p, "reg", 0)),
                  int(getattr(p, "tv_iters", 10)))


def reconstruct(g: Geom, counts, gamma, params, f0, nsub: int = -1, with_objective=False,
                mult=None):
    """Run SDP-BSREM (Table I) for ``nsub`` subiterations (all T M when -1); with ``mult``
    ([P][V][n_b] float32) the system matrix is diag(mult) A.

    Returns (f, objective history or None)."""
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    gamma = np.ascontiguousarray(gamma, dtype=np.float32)
    keep, mp = _fptr(mult)
    f = np.array(f0, dtype=np.float64, copy=True, order="C")
    prm = params if isinstance(params, Params) else params_from(params)
    obj = np.full(prm.iterations + 1, np.nan) if with_objective else None
    lib().ora_reconstruct_m(ctypes.byref(g), counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            gamma.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), mp,
                            ctypes.byref(prm), f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            nsub,
                            obj.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if obj is not None else None,
                            None)
    return f, obj


def reconstruct_snapshots(g: Geom, counts, gamma, params, f0):
    """Full run (T iterations) returning (f after each iteration [T][P][N][N], objective T+1)."""
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    gamma = np.ascontiguousarray(gamma, dtype=np.float32)
    f = np.array(f0, dtype=np.float64, copy=True, order="C")
    prm = params if isinstance(params, Params) else params_from(params)
    obj = np.full(prm.iterations + 1, np.nan)
    snaps = np.zeros((prm.iterations,) + f.shape)
    lib().ora_reconstruct_snap(ctypes.byref(g), counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               gamma.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(prm),
                               f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), -1,
                               obj.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               snaps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return snaps, obj
