"""Thin ctypes binding of libpet (declared in include/pet.h).

Argument marshalling only: every function forwards torch tensors' device pointers (or numpy
host buffers) to the C ABI of the same name, and raises ``PetError`` on a non-OK status.  All
computation happens in the CUDA library; there is no fallback: if ``libpet.so`` is missing
or cannot be loaded, importing a function raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpet.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, PENDING, ERR_NOT_FOUND = range(7)
PRECOND = dict(BSREM=0, M1=1, M2=2, P1=3, P2=4)
PREC_FP32, PREC_FP32_KAHAN, PREC_FP64 = 0, 1, 2


class PetError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libpet status {status}: {msg}")
        self.status = status


class GeometryDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nplanes", ctypes.c_int), ("pixel_mm", ctypes.c_double),
                ("nviews", ctypes.c_int), ("nbins", ctypes.c_int), ("bin_mm", ctypes.c_double),
                ("nsubsets", ctypes.c_int), ("sens", ctypes.c_double), ("subrays", ctypes.c_int),
                ("tof_bins", ctypes.c_int), ("tof_bin_mm", ctypes.c_double),
                ("tof_fwhm_mm", ctypes.c_double), ("ring_mm", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int)] + [
        (k, ctypes.c_double) for k in ("beta", "gamma_r", "eps", "t", "U", "lambda0", "a",
                                       "rho", "delta1", "delta2", "nu1", "nu2")] + [
        ("J0", ctypes.c_int), ("J1", ctypes.c_int), ("precond", ctypes.c_int),
        ("precision", ctypes.c_int), ("rdp_3d", ctypes.c_int), ("regularizer", ctypes.c_int),
        ("tv_iters", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("geom", GeometryDesc), ("h_counts", ctypes.c_void_p), ("h_gamma", ctypes.c_void_p),
                ("h_img_init", ctypes.c_void_p), ("params", Params), ("with_objective", ctypes.c_int),
                ("h_mult", ctypes.c_void_p)]


class ServeStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longlong) for k in ("submitted", "completed", "failed", "running", "queued")] + [
        (k, ctypes.c_double) for k in ("p50_s", "p99_s", "mean_s", "scans_per_s")] + [
        ("hbm_in_use", ctypes.c_size_t)] + [
        (k, ctypes.c_double) for k in ("mean_queue_s", "mean_prepare_s", "mean_run_s",
                                       "mean_readback_s")] + [
        ("tuned_geometries", ctypes.c_longlong)]


_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes)
SIGNATURES = {
    "pet_last_error": (ctypes.c_char_p, []),
    "pet_geometry_create": (_I, [ctypes.POINTER(GeometryDesc), _VP, ctypes.POINTER(_VP)]),
    "pet_geometry_destroy": (None, [_VP]),
    "pet_subset_size": (_I, [_VP, _I]),
    "pet_autotune": (_I, [_VP, _VP, ctypes.POINTER(_I)]),
    "pet_autotune_batch": (_I, [_VP, _I, _VP, ctypes.POINTER(_I)]),
    "pet_set_ray_chunks": (_I, [_VP, _I]),
    "pet_sensitivity": (_I, [_VP, _VP, _VP]),
    "pet_forward_subset": (_I, [_VP, _I, _VP, _VP, _VP]),
    "pet_back_subset": (_I, [_VP, _I, _VP, _VP, _VP]),
    "pet_forward_subset_f64": (_I, [_VP, _I, _VP, _VP, _VP]),
    "pet_back_subset_f64": (_I, [_VP, _I, _VP, _VP, _VP]),
    "pet_debug_fail_alloc": (None, [ctypes.c_int]),
    "pet_debug_bp_table": (None, [ctypes.c_int]),
    "pet_state_create": (_I, [_VP, _VP, _VP, ctypes.POINTER(Params), _VP, _VP, ctypes.POINTER(_VP)]),
    "pet_state_create_attn": (_I, [_VP, _VP, _VP, _VP, ctypes.POINTER(Params), _VP, _VP,
                                   ctypes.POINTER(_VP)]),
    "pet_subiter": (_I, [_VP, _VP]),
    "pet_state_read_image": (_I, [_VP, _VP, _VP]),
    "pet_state_read_image_f64": (_I, [_VP, _VP, _VP]),
    "pet_state_objective": (_I, [_VP, _DP, _DP, _VP]),
    "pet_state_subiters": (_I, [_VP]),
    "pet_state_export": (_I, [_VP, _VP, ctypes.POINTER(ctypes.c_size_t), _VP]),
    "pet_state_import": (_I, [_VP, _VP, ctypes.c_size_t, _VP]),
    "pet_state_reset": (_I, [_VP, _VP, _VP]),
    "pet_state_destroy": (None, [_VP]),
    "pet_reconstruct": (_I, [_VP, _VP, _VP, ctypes.POINTER(Params), _VP, _DP, _VP]),
    "pet_reconstruct_attn": (_I, [_VP, _VP, _VP, _VP, ctypes.POINTER(Params), _VP, _DP, _VP]),
    "pet_reconstruct_host": (_I, [_VP, _VP, _VP, ctypes.POINTER(Params), _VP, _DP, _VP]),
    "pet_rdp_gradient": (_I, [_VP, _VP, _D, _D, _VP, _VP]),
    "pet_smoothness_nu": (_I, [_VP, _VP, _D, _D, _VP, _VP]),
    "pet_objective": (_I, [_VP, _VP, _VP, _VP, _D, _D, _D, _DP, _DP, _VP]),
    "pet_objective_static": (_I, [_VP, _VP, _VP, _VP, _D, _D, _D, _DP, _DP, _VP]),
    "pet_rdp_gradient_3d": (_I, [_VP, _VP, _D, _D, _VP, _VP]),
    "pet_smoothness_nu_3d": (_I, [_VP, _VP, _D, _D, _VP, _VP]),
    "pet_objective_3d": (_I, [_VP, _VP, _VP, _VP, _D, _D, _D, _DP, _DP, _VP]),
    "pet_objective_tv": (_I, [_VP, _VP, _VP, _VP, _D, _DP, _DP, _VP]),
    "pet_tv_prox": (_I, [_VP, _VP, _VP, _D, _I, _VP, _VP, _VP, _VP]),
    "pet_batch_create": (_I, [_I, _I, ctypes.POINTER(_VP)]),
    "pet_batch_add": (_I, [_VP, _VP, _I, _VP]),
    "pet_batch_remove": (_I, [_VP, _VP]),
    "pet_batch_step": (_I, [_VP, _VP, ctypes.POINTER(_I)]),
    "pet_batch_size": (_I, [_VP]),
    "pet_batch_destroy": (None, [_VP]),
    "pet_state_objective_history": (_I, [_VP, _DP, _VP]),
    "pet_serve_create": (_I, [ctypes.c_size_t, _I, _I, ctypes.POINTER(_VP)]),
    "pet_serve_submit": (_I, [_VP, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "pet_serve_poll": (_I, [_VP, ctypes.c_uint64, _VP, _DP, _DP]),
    "pet_serve_stats_get": (_I, [_VP, ctypes.POINTER(ServeStats)]),
    "pet_serve_destroy": (None, [_VP]),
    "pet_serve_autotune": (_I, [_VP, _I]),
    "pet_launch_count": (ctypes.c_longlong, []),
    "pet_profile_enable": (None, [_I]),
    "pet_profile_read": (_I, [_I, _DP, ctypes.POINTER(ctypes.c_longlong)]),
    "pet_profile_reset": (None, []),
}

KERNEL_KINDS = ["forward_ratio", "update", "mu_sum", "obj_forward", "rdp_value", "layout", "other"]


def lib():
    """Load libpet.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise PetError(ERR_CUDA, f"{LIB_PATH} is not built; run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def debug_fail_alloc(n: int):
    """Test hook: the n-th device / pinned allocation of the library from now fails as out of
    memory (n <= 0 disarms); host-side fault injection."""
    lib().pet_debug_fail_alloc(int(n))


def debug_bp_table(enable: bool):
    """Test hook: geometries created from now on skip (False) or build (True, the default) the
    precomputed backprojection entries of the FP32 update; the results are the same bits."""
    lib().pet_debug_bp_table(1 if enable else 0)


def _check(status: int):
    if status != OK:
        raise PetError(status, lib().pet_last_error().decode())


def _ptr(t) -> int | None:
    """Device pointer of a torch tensor (contiguous), host pointer of a numpy array."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        assert t.is_contiguous(), "tensors passed to libpet must be contiguous"
        return t.data_ptr()
    assert t.flags["C_CONTIGUOUS"], "arrays passed to libpet must be C-contiguous"
    return t.ctypes.data


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def make_params(p, precision: int | None = None) -> Params:
    """Params from an object with AlgoParams attribute names."""
    return Params(p.iterations, p.beta, p.gamma_r, p.eps, p.t, p.U, p.lambda0, p.a, p.rho,
                  p.delta1, p.delta2, p.nu1, p.nu2, p.J0, p.J1, p.precond,
                  p.precision if precision is None else precision, int(getattr(p, "rdp3d", 0)),
                  int(getattr(p, "reg", 0)), int(getattr(p, "tv_iters", 10)))


class Geometry:
    """pet_geometry handle (Sec. II-A/B geometry, subsets, sensitivity)."""

    def __init__(self, n, nplanes, pixel_mm, nviews, nbins, bin_mm, nsubsets, sens, stream=None,
                 subrays=1, tof_bins=0, tof_bin_mm=0.0, tof_fwhm_mm=0.0, ring_mm=0.0):
        self.desc = GeometryDesc(n, nplanes, pixel_mm, nviews, nbins, bin_mm, nsubsets, sens, subrays,
                                 tof_bins, tof_bin_mm, tof_fwhm_mm, ring_mm)
        self.tof_bins = max(1, tof_bins)
        h = _VP()
        _check(lib().pet_geometry_create(ctypes.byref(self.desc), _stream(stream), ctypes.byref(h)))
        self.handle = h
        self.n, self.nplanes, self.nviews, self.nbins, self.nsubsets = n, nplanes, nviews, nbins, nsubsets

    @classmethod
    def from_dict(cls, geometry: dict, sens: float, stream=None):
        g = geometry
        return cls(g["n"], g["nplanes"], g["pixel_mm"], g["nviews"], g["nbins"], g["bin_mm"],
                   g["nsubsets"], sens, stream, int(g.get("subrays", 1)), int(g.get("tof_bins", 0)),
                   float(g.get("tof_bin_mm", 0.0)), float(g.get("tof_fwhm_mm", 0.0)),
                   float(g.get("ring_mm", 0.0)))

    def close(self):
        if getattr(self, "handle", None):
            lib().pet_geometry_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def subset_size(self, subset: int) -> int:
        return lib().pet_subset_size(self.handle, subset)

    def autotune(self, stream=None) -> int:
        """Pick the forward projector's ray chunking by timing it; returns the chosen value."""
        s = ctypes.c_int()
        _check(lib().pet_autotune(self.handle, _stream(stream), ctypes.byref(s)))
        return s.value

    def autotune_batch(self, concurrent: int, stream=None) -> int:
        """Pick the ray chunking with `concurrent` projections sharing the GPU (batched scans)."""
        s = ctypes.c_int()
        _check(lib().pet_autotune_batch(self.handle, int(concurrent), _stream(stream), ctypes.byref(s)))
        return s.value

    def set_ray_chunks(self, S: int):
        """Fix the forward projector's ray chunks (0: built-in heuristic)."""
        _check(lib().pet_set_ray_chunks(self.handle, int(S)))


def sensitivity(g: Geometry, d_p, stream=None):
    _check(lib().pet_sensitivity(g.handle, _ptr(d_p), _stream(stream)))


def forward_subset(g: Geometry, subset: int, d_img, d_proj, stream=None):
    fn = lib().pet_forward_subset_f64 if str(d_img.dtype) == "torch.float64" else lib().pet_forward_subset
    _check(fn(g.handle, subset, _ptr(d_img), _ptr(d_proj), _stream(stream)))


def back_subset(g: Geometry, subset: int, d_proj, d_img, stream=None):
    fn = lib().pet_back_subset_f64 if str(d_proj.dtype) == "torch.float64" else lib().pet_back_subset
    _check(fn(g.handle, subset, _ptr(d_proj), _ptr(d_img), _stream(stream)))


class State:
    """pet_state handle: resident reconstruction state (Table I)."""

    def __init__(self, g: Geometry, d_counts, d_gamma, params: Params, d_img_init, stream=None,
                 d_mult=None):
        """d_mult: per-bin detection factors (float32 [P][V][NB], device) for the system matrix
        diag(a) A (pet_state_create_attn), or None."""
        h = _VP()
        self.params = params
        if d_mult is None:
            _check(lib().pet_state_create(g.handle, _ptr(d_counts), _ptr(d_gamma), ctypes.byref(params),
                                          _ptr(d_img_init), _stream(stream), ctypes.byref(h)))
        else:
            _check(lib().pet_state_create_attn(g.handle, _ptr(d_counts), _ptr(d_gamma), _ptr(d_mult),
                                               ctypes.byref(params), _ptr(d_img_init), _stream(stream),
                                               ctypes.byref(h)))
        self.handle = h

    def subiter(self, stream=None):
        _check(lib().pet_subiter(self.handle, _stream(stream)))

    def reset(self, d_img_init=None, stream=None):
        _check(lib().pet_state_reset(self.handle, _ptr(d_img_init), _stream(stream)))

    def read_image(self, d_img, stream=None):
        fn = lib().pet_state_read_image_f64 if str(d_img.dtype) == "torch.float64" else lib().pet_state_read_image
        _check(fn(self.handle, _ptr(d_img), _stream(stream)))

    def objective(self, stream=None):
        phi = ctypes.c_double()
        parts = (ctypes.c_double * 3)()
        _check(lib().pet_state_objective(self.handle, ctypes.byref(phi), parts, _stream(stream)))
        return phi.value, list(parts)

    @property
    def subiters(self) -> int:
        return lib().pet_state_subiters(self.handle)

    def export(self, stream=None) -> bytes:
        """The state's checkpoint (host bytes)."""
        n = ctypes.c_size_t()
        _check(lib().pet_state_export(self.handle, None, ctypes.byref(n), _stream(stream)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().pet_state_export(self.handle, buf, ctypes.byref(n), _stream(stream)))
        return buf.raw[:n.value]

    def load(self, blob: bytes, stream=None):
        """Resume from a checkpoint written by export() for the same geometry and parameters."""
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().pet_state_import(self.handle, buf, len(blob), _stream(stream)))

    def objective_history(self, stream=None):
        """Phi(f^k), k = 0..T, recorded so far (NaN where not computed)."""
        out = (ctypes.c_double * (self.params.iterations + 1))()
        _check(lib().pet_state_objective_history(self.handle, out, _stream(stream)))
        return list(out)

    def close(self):
        if getattr(self, "handle", None):
            lib().pet_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reconstruct(g: Geometry, d_counts, d_gamma, params: Params, d_img_inout, objective=False,
                stream=None, d_mult=None):
    """f^0 -> f^T in place; returns the objective history (T+1 values) if requested.  d_mult:
    per-bin detection factors (pet_reconstruct_attn), or None."""
    obj = (ctypes.c_double * (params.iterations + 1))() if objective else None
    if d_mult is None:
        _check(lib().pet_reconstruct(g.handle, _ptr(d_counts), _ptr(d_gamma), ctypes.byref(params),
                                     _ptr(d_img_inout), obj, _stream(stream)))
    else:
        _check(lib().pet_reconstruct_attn(g.handle, _ptr(d_counts), _ptr(d_gamma), _ptr(d_mult),
                                          ctypes.byref(params), _ptr(d_img_inout), obj,
                                          _stream(stream)))
    return list(obj) if objective else None


def reconstruct_host(g: Geometry, h_counts, h_gamma, params: Params, h_img_inout, objective=False,
                     stream=None):
    """Host-buffer variant (numpy or pinned CPU tensors); copies happen inside the call."""
    obj = (ctypes.c_double * (params.iterations + 1))() if objective else None
    _check(lib().pet_reconstruct_host(g.handle, _ptr(h_counts), _ptr(h_gamma), ctypes.byref(params),
                                      _ptr(h_img_inout), obj, _stream(stream)))
    return list(obj) if objective else None


def rdp_gradient(g: Geometry, d_img, gamma_r, eps, d_grad, stream=None, three_d=False):
    fn = lib().pet_rdp_gradient_3d if three_d else lib().pet_rdp_gradient
    _check(fn(g.handle, _ptr(d_img), gamma_r, eps, _ptr(d_grad), _stream(stream)))


def smoothness_nu(g: Geometry, d_img, nu1, nu2, d_nu, stream=None, three_d=False):
    fn = lib().pet_smoothness_nu_3d if three_d else lib().pet_smoothness_nu
    _check(fn(g.handle, _ptr(d_img), nu1, nu2, _ptr(d_nu), _stream(stream)))


def objective(g: Geometry, d_counts, d_gamma, d_img, beta, gamma_r, eps, stream=None, three_d=False):
    phi = ctypes.c_double()
    parts = (ctypes.c_double * 3)()
    fn = lib().pet_objective_3d if three_d else lib().pet_objective
    _check(fn(g.handle, _ptr(d_counts), _ptr(d_gamma), _ptr(d_img), beta, gamma_r,
              eps, ctypes.byref(phi), parts, _stream(stream)))
    return phi.value, list(parts)


def objective_tv(g: Geometry, d_counts, d_gamma, d_img, beta, stream=None):
    """Phi with the TV variant's R_TV (parts[2] = R_TV(d_img))."""
    phi = ctypes.c_double()
    parts = (ctypes.c_double * 3)()
    _check(lib().pet_objective_tv(g.handle, _ptr(d_counts), _ptr(d_gamma), _ptr(d_img), beta,
                                  ctypes.byref(phi), parts, _stream(stream)))
    return phi.value, list(parts)


def tv_prox(g: Geometry, d_z, d_w, b, iters, d_px, d_py, d_x, stream=None):
    """The TV variant's proximal step (primal-dual iterations); d_px, d_py updated in place."""
    _check(lib().pet_tv_prox(g.handle, _ptr(d_z), _ptr(d_w), float(b), int(iters), _ptr(d_px),
                             _ptr(d_py), _ptr(d_x), _stream(stream)))


def objective_static(g: Geometry, d_counts, d_gamma, d_img, beta, gamma_r, eps, stream=None):
    """Phi(d_img) like ``objective``, through the entry point that allocates no memory."""
    phi = ctypes.c_double()
    parts = (ctypes.c_double * 3)()
    _check(lib().pet_objective_static(g.handle, _ptr(d_counts), _ptr(d_gamma), _ptr(d_img), beta,
                                      gamma_r, eps, ctypes.byref(phi), parts, _stream(stream)))
    return phi.value, list(parts)


def launch_count() -> int:
    return lib().pet_launch_count()


def profile_enable(on: bool = True):
    lib().pet_profile_enable(1 if on else 0)


def profile_reset():
    lib().pet_profile_reset()


def profile_read() -> dict:
    """{kind: (total device ms, launches)} for every kernel kind (synchronises)."""
    out = {}
    for k, name in enumerate(KERNEL_KINDS):
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        _check(lib().pet_profile_read(k, ctypes.byref(ms), ctypes.byref(n)))
        out[name] = (ms.value, n.value)
    return out


class Batch:
    """pet_batch: many states advanced together by batched, graph-replayed kernels."""

    def __init__(self, capacity: int, use_graph: bool = True):
        h = _VP()
        _check(lib().pet_batch_create(capacity, 1 if use_graph else 0, ctypes.byref(h)))
        self.handle = h
        self.members = []

    def add(self, state: State, with_objective: bool = False, stream=None):
        _check(lib().pet_batch_add(self.handle, state.handle, 1 if with_objective else 0, _stream(stream)))
        self.members.append(state)

    def remove(self, state: State):
        _check(lib().pet_batch_remove(self.handle, state.handle))
        self.members.remove(state)

    def step(self, stream=None) -> int:
        n = ctypes.c_int()
        _check(lib().pet_batch_step(self.handle, _stream(stream), ctypes.byref(n)))
        return n.value

    @property
    def running(self) -> int:
        return lib().pet_batch_size(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            lib().pet_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """pet_server: continuous batching of reconstruction requests (host buffers in and out)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int, device: int = 0):
        h = _VP()
        _check(lib().pet_serve_create(int(hbm_budget_bytes), max_slots, device, ctypes.byref(h)))
        self.handle = h
        self.shapes = {}

    def submit(self, geometry: dict, sens: float, counts, gamma, params: Params, img0=None,
               with_objective: bool = True, mult=None) -> int:
        """mult: per-bin detection factors ([P][V][n_b] float32, host) or None."""
        import numpy as np
        g = geometry
        desc = GeometryDesc(g["n"], g["nplanes"], g["pixel_mm"], g["nviews"], g["nbins"], g["bin_mm"],
                            g["nsubsets"], sens, int(g.get("subrays", 1)), int(g.get("tof_bins", 0)),
                            float(g.get("tof_bin_mm", 0.0)), float(g.get("tof_fwhm_mm", 0.0)),
                            float(g.get("ring_mm", 0.0)))
        counts = np.ascontiguousarray(counts, dtype=np.int32)
        gamma = np.ascontiguousarray(gamma, dtype=np.float32)
        img0 = None if img0 is None else np.ascontiguousarray(img0, dtype=np.float32)
        mult = None if mult is None else np.ascontiguousarray(mult, dtype=np.float32)
        req = Request(desc, counts.ctypes.data, gamma.ctypes.data,
                      None if img0 is None else img0.ctypes.data, params, 1 if with_objective else 0,
                      None if mult is None else mult.ctypes.data)
        t = ctypes.c_uint64()
        _check(lib().pet_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        self.shapes[t.value] = ((g["nplanes"], g["n"], g["n"]), params.iterations + 1)
        return t.value

    def poll(self, ticket: int):
        """None while pending; else (image [P][N][N] float32, objective list, latency_s)."""
        import numpy as np
        shape, nobj = self.shapes.get(ticket, ((0,), 1))
        img = np.empty(shape, np.float32)
        obj = (ctypes.c_double * nobj)()
        lat = ctypes.c_double()
        st = lib().pet_serve_poll(self.handle, ticket, img.ctypes.data if img.size else None,
                                  obj, ctypes.byref(lat))
        if st == PENDING:
            return None
        self.shapes.pop(ticket, None)
        _check(st)
        return img, list(obj), lat.value

    def autotune(self, concurrent: int):
        """Tune every new geometry for `concurrent` scans sharing the GPU (0: built-in shapes)."""
        _check(lib().pet_serve_autotune(self.handle, int(concurrent)))

    def stats(self) -> dict:
        s = ServeStats()
        _check(lib().pet_serve_stats_get(self.handle, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ServeStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().pet_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
